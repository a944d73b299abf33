// lmf_kernels.cu -- view build, plain root scan, combine and finalize kernels.
//
// Step map (method -> kernel):
//   child views, Sec. 3.2 (directional views) and Ex. 3.1     -> k_view_unique / k_view_general
//   merged views probed at the root, Sec. 3.4 case (1)        -> GroupDesc records
//   one scan of the root with view lookups, Sec. 3.5          -> k_root_plain (and lmf_gram_tc.cu)
//   covar entries SUM(x_i x_j), Eq. lr-sigma of Sec. 2        -> Gram of z = [1, x, view means]
//   grouped covar entries Covar(X_j; X_k), Covar(X_j, X_k; 1) -> reverse views + k_rv_tasks / DirectAgg
//   cross-block combine and placement                          -> k_combine, k_corr, k_out_map
#include "lmf_internal.h"
#include "lmf_root_plain.cuh"
#include "lmf_rowpass.cuh"

#include <algorithm>
#include <cstdint>
#include <cstdio>

namespace lmf {

// ---------------------------------------------------------------------------
// helpers
__device__ __forceinline__ float load_f(const Col& c, int64_t i) {
  return c.dtype == 2 ? static_cast<float>(static_cast<const double*>(c.p)[i])
                      : static_cast<const float*>(c.p)[i];
}
__device__ __forceinline__ double load_d(const Col& c, int64_t i) {
  return c.dtype == 2 ? static_cast<const double*>(c.p)[i]
                      : static_cast<double>(static_cast<const float*>(c.p)[i]);
}
__device__ __forceinline__ void add_ll(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}
// exact fixed-point image of w * x: x * scale is a power-of-two scaling of a
// float (exact unless it underflows), its integer part is taken with rounding
__device__ __forceinline__ long long fixp(long long w, float x, float scale) {
  return w * __float2ll_rn(x * scale);
}

// ---------------------------------------------------------------------------
// A1: key statistics and value ranges (declare / plan time)
__global__ void k_minmax_i32(const int32_t* key, int64_t n, int* mm) {
  int lo = 0x7fffffff, hi = -0x7fffffff - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int v = key[i];
    lo = min(lo, v);
    hi = max(hi, v);
  }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(mm, lo);
    atomicMax(mm + 1, hi);
  }
}

__global__ void k_hist_i32(const int32_t* key, int64_t n, unsigned int* hist, int K) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int v = key[i];
    if (v >= 0 && v < K) atomicAdd(hist + v, 1u);
  }
}

cudaError_t launch_key_stats(const int32_t* key, int64_t n, unsigned int* hist, int K, int* minmax,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t gb = (n + 255) / 256;
  int grid = (int)(gb < 4096 ? gb : 4096);
  if (hist == nullptr) {
    k_minmax_i32<<<grid, 256, 0, s>>>(key, n, minmax);
  } else {
    k_hist_i32<<<grid, 256, 0, s>>>(key, n, hist, K);
  }
  return cudaGetLastError();
}

// number of i in [1, n) with key[i] != key[i - 1]: one less than the runs of
// equal keys
__global__ void k_key_changes(const int32_t* key, int64_t n, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += key[i] != key[i - 1];
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_key_changes(const int32_t* key, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  int64_t gb = (n + 255) / 256;
  int grid = (int)(gb < 2048 ? gb : 2048);
  k_key_changes<<<grid, 256, 0, s>>>(key, n, out);
  return cudaGetLastError();
}

__global__ void k_colmaxabs(const Col c, int64_t n, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = fabs(load_d(c, i));
    m = v > m ? v : m;  // NaN is dropped
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
}

cudaError_t launch_colmaxabs(const Col* cols, int n, int64_t nrows, double* out, cudaStream_t s) {
  for (int i = 0; i < n; ++i) {
    if (nrows <= 0) continue;
    int64_t gb = (nrows + 255) / 256;
    int grid = (int)(gb < 2048 ? gb : 2048);
    k_colmaxabs<<<grid, 256, 0, s>>>(cols[i], nrows, reinterpret_cast<unsigned long long*>(out + i));
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A2: child views, unique keys (every key has at most one row and every
// subtree count is 0 or 1): the record of key k is written by its one row.
__global__ void k_view_unique(const __grid_constant__ ViewArgs a) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.nrows) return;
  const int32_t k = a.key[row];
  if (k < 0) return;  // a negative key joins no parent row
  if (k >= a.K) {
    atomicOr(a.status, kStatusKeyRange);
    return;
  }
  uint32_t* dst = a.dst + (int64_t)k * a.dst_stride;
  long long cnt = 1;
  int mu = a.mu_off, cat = a.cat_off;
  for (int i = 0; i < a.n_own; ++i) dst[mu++] = __float_as_uint(load_f(a.own[i], row));
  for (int i = 0; i < a.n_owncat; ++i) {
    int32_t v = a.owncat[i][row];
    if (v < 0 || v >= a.owncat_dom[i]) {
      atomicOr(a.status, kStatusCatRange);
      v = 0;
    }
    dst[cat++] = static_cast<uint32_t>(v);
  }
  for (int g = 0; g < a.n_grp; ++g) {
    const GroupDesc& G = a.grp[g];
    const int32_t fk = G.fk[row];
    const bool hit = fk >= 0 && fk < G.K;
    const uint32_t* rec = G.rec + (hit ? (int64_t)fk * G.stride : 0);
    for (int c = 0; c < G.n_cnt; ++c) cnt *= hit ? static_cast<long long>(rec[c]) : 0;
    for (int j = 0; j < G.n_mu; ++j) dst[mu++] = hit ? rec[G.n_cnt + j] : 0u;
    for (int j = 0; j < G.n_cat; ++j) dst[cat++] = hit ? rec[G.n_cnt + G.n_mu + j] : 0u;
  }
  dst[a.cnt_word] = static_cast<uint32_t>(cnt);
}

cudaError_t launch_view_unique(const ViewArgs& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  k_view_unique<<<(unsigned)((a.nrows + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// A2, general keys: subtree counts, sums and second moments per key, in
// exact fixed-point integers (order-independent, so deterministic).  With
// e's subtree count c_e and within-key scatter Sc_e, a row's contribution to
// its key is  c * xt xt^T  +  sum_e (c / c_e) * Sc_e  (placed on e's block),
// c = prod_e c_e, xt = [own features, means of the children's subtrees].
__device__ __forceinline__ int tri_index(int i, int j, int d) {  // i <= j
  return i * d - i * (i - 1) / 2 + (j - i);
}

__global__ void k_view_general(const __grid_constant__ ViewArgs a) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.nrows) return;
  const int32_t k = a.key[row];
  if (k < 0) return;  // a negative key joins no parent row
  if (k >= a.K) {
    atomicOr(a.status, kStatusKeyRange);
    return;
  }
  double xt[kMaxZ];
  long long wc[kMaxGroups * 4];
  int nwc = 0;
  int d = 0;
  for (int i = 0; i < a.n_own; ++i) xt[d++] = load_d(a.own[i], row);
  long long cnt = 1;
  const uint32_t* recs[kMaxGroups];
  int32_t fks[kMaxGroups];
  for (int g = 0; g < a.n_grp; ++g) {
    const GroupDesc& G = a.grp[g];
    const int32_t fk = G.fk[row];
    const bool hit = fk >= 0 && fk < G.K;
    fks[g] = hit ? fk : -1;
    recs[g] = hit ? G.rec + (int64_t)fk * G.stride : nullptr;
    for (int c = 0; c < G.n_cnt; ++c) {
      long long v = hit ? static_cast<long long>(recs[g][c]) : 0;
      wc[nwc++] = v;
      cnt *= v;
    }
    for (int j = 0; j < G.n_mu; ++j) xt[d++] = hit ? (double)__uint_as_float(recs[g][G.n_cnt + j]) : 0.0;
  }
  if (cnt == 0) return;
  add_ll(reinterpret_cast<long long*>(a.cnt64 + k), cnt);
  long long* S = a.S + (int64_t)k * a.d;
  long long* Q = a.Q + (int64_t)k * a.dq;
  const double c = static_cast<double>(cnt);
  for (int i = 0; i < a.d; ++i) add_ll(S + i, llrint(c * xt[i] * (double)a.s_scale[i]));
  for (int i = 0; i < a.d; ++i)
    for (int j = i; j < a.d; ++j) add_ll(Q + tri_index(i, j, a.d), llrint(c * xt[i] * xt[j] * a.q_scale));
  // scatter of fanning-out grandchildren, weighted by the other counts
  int wbase[kMaxGroups + 1];
  wbase[0] = 0;
  for (int g = 0; g < a.n_grp; ++g) wbase[g + 1] = wbase[g] + a.grp[g].n_cnt;
  for (int e = 0; e < a.n_sc; ++e) {
    const int g = a.sc_grp[e];
    if (fks[g] < 0) continue;
    long long other = 1;
    const int self = wbase[g] + a.sc_cntword[e];
    for (int q = 0; q < nwc; ++q)
      if (q != self) other *= wc[q];
    const int de = a.sc_d[e], f0 = a.sc_feat0[e];
    const double* sc = a.sc[e] + (int64_t)fks[g] * (de * (de + 1) / 2);
    for (int i = 0; i < de; ++i)
      for (int j = i; j < de; ++j)
        add_ll(Q + tri_index(f0 + i, f0 + j, a.d),
               llrint((double)other * sc[tri_index(i, j, de)] * a.q_scale));
  }
}

cudaError_t launch_view_general(const ViewArgs& a, cudaStream_t s) {
  if (a.nrows <= 0) return cudaSuccess;
  k_view_general<<<(unsigned)((a.nrows + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

__global__ void k_view_finalize(const __grid_constant__ ViewFinalizeArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  const unsigned long long c = a.cnt64[k];
  uint32_t* dst = a.dst + (int64_t)k * a.dst_stride;
  if (c > 0x7fffffffull) atomicOr(a.status, kStatusOverflow);
  dst[a.cnt_word] = static_cast<uint32_t>(c > 0x7fffffffull ? 0x7fffffffull : c);
  double s[kMaxZ];
  for (int i = 0; i < a.d; ++i) {
    s[i] = c ? (double)a.S[(int64_t)k * a.d + i] / (double)a.s_scale[i] : 0.0;
    dst[a.mu_off + i] = __float_as_uint(c ? (float)(s[i] / (double)c) : 0.f);
  }
  double* sc = a.sc + (int64_t)k * a.dq;
  for (int i = 0; i < a.d; ++i)
    for (int j = i; j < a.d; ++j) {
      const int t = tri_index(i, j, a.d);
      sc[t] = c ? (double)a.Q[(int64_t)k * a.dq + t] / a.q_scale - s[i] * s[j] / (double)c : 0.0;
    }
}

cudaError_t launch_view_finalize(const ViewFinalizeArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_view_finalize<<<(a.K + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A3-A5: the plain root scan (body in lmf_root_plain.cuh) with the generic
// row pass
template <int MP>
__global__ void __launch_bounds__(256) k_root_plain(const __grid_constant__ RootParams p, int64_t n_tiles) {
  root_plain_body<MP, GenericRowPass>(p, n_tiles);
}

size_t root_plain_smem(int mp, int n_rowcat, int cache_cells, int res_cells, bool unit_w) {
  size_t z = (size_t)(unit_w ? 1 : 2) * kPlainT * (mp + 4) * sizeof(float);
  size_t c = (size_t)kPlainT * (n_rowcat > 0 ? n_rowcat : 1) * sizeof(int32_t);
  const size_t nbk = mp / 4, nb = nbk * (nbk + 1) / 2, rg = nb >= 256 ? 1 : 256 / nb;
  const size_t red = nb * 16 * rg * sizeof(double);  // the final reduction's scratch
  const size_t total = z + c + (size_t)(cache_cells + res_cells) * 4;
  return total > red ? total : red;
}
int root_plain_tile_rows() { return kPlainT; }

template <int MP>
static cudaError_t launch_plain_mp(const RootParams& p, int grid, int64_t n_tiles, size_t smem,
                                   cudaStream_t s) {
  k_root_plain<MP><<<grid, 256, smem, s>>>(p, n_tiles);
  return cudaGetLastError();
}

cudaError_t root_plain_prepare(int mp, size_t smem) {
  const int v = (int)smem;
  switch (mp) {
    case 16: return cudaFuncSetAttribute(k_root_plain<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    case 32: return cudaFuncSetAttribute(k_root_plain<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    case 48: return cudaFuncSetAttribute(k_root_plain<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    case 64: return cudaFuncSetAttribute(k_root_plain<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_root_plain(const RootParams& p, int mp, int grid, int64_t n_tiles, size_t smem,
                              cudaStream_t s) {
  switch (mp) {
    case 16: return launch_plain_mp<16>(p, grid, n_tiles, smem, s);
    case 32: return launch_plain_mp<32>(p, grid, n_tiles, smem, s);
    case 48: return launch_plain_mp<48>(p, grid, n_tiles, smem, s);
    case 64: return launch_plain_mp<64>(p, grid, n_tiles, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// A9: ordered FP64 combine of the per-CTA partials (deterministic)
// the partials cover z[off, off + n): entry (i, j) of a CTA's block lands at
// G[off + i][off + j]
// one warp per entry (i <= j), lanes striding over the CTAs, a fixed shuffle
// tree: the same order on every run
__global__ void k_combine(const double* part, int grid, int mp, int m, const long long* cnt_part,
                          double* G, long long* count, int off, int n) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (e < n * n) {
    const int i = e / n, j = e % n;
    if (i <= j) {
      double s = 0.0;
      for (int c = lane; c < grid; c += 32) s += part[(int64_t)c * mp * mp + i * mp + j];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        G[(off + i) * m + off + j] = s;
        G[(off + j) * m + off + i] = s;
      }
    }
  } else if (e == n * n) {
    long long s = 0;
    for (int c = lane; c < grid; c += 32) s += cnt_part[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *count = s;
  }
}

cudaError_t launch_combine(const double* part, int grid, int mp, int m, const long long* cnt_part,
                           double* G, long long* count, cudaStream_t s, int off, int n) {
  if (n < 0) n = m;
  const int warps = n * n + 1;  // the last one sums the counts
  k_combine<<<(warps + 3) / 4, 128, 0, s>>>(part, grid, mp, m, cnt_part, G, count, off, n);
  return cudaGetLastError();
}

__global__ void k_corr(const CorrTask* tasks, double* G, int m) {
  const CorrTask t = tasks[blockIdx.x];
  const int dq = t.d * (t.d + 1) / 2;
  for (int e = threadIdx.x; e < dq; e += blockDim.x) {
    int i = 0, r = e;
    while (r >= t.d - i) {
      r -= t.d - i;
      ++i;
    }
    const int j = i + r;
    double s = 0.0;
    for (int k = 0; k < t.K; ++k) s += (double)t.omega[k] * t.sc[(int64_t)k * dq + e];
    const int a = t.zoff + i, b = t.zoff + j;
    G[a * m + b] += s;
    if (a != b) G[b * m + a] += s;
  }
}

cudaError_t launch_corr(const void* tasks_dev, int n, double* G, int m, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_corr<<<n, 128, 0, s>>>(static_cast<const CorrTask*>(tasks_dev), G, m);
  return cudaGetLastError();
}

// grouped aggregates answered from a reverse view: one pass over the group's
// keys, every task of the view served from the key's record and slots
// round(c * m * scale) for a count c < 2^40, an FP32 value m and a power-of-two
// scale, exactly, in integer arithmetic: m = M 2^(e - 150) with the 24-bit
// integer M, so c m scale = (c M) 2^sh, c M exact in 64 bits, then one
// rounding (half away from zero) by the shift.  The plan's scale keeps the
// result below 2^62.
__device__ __forceinline__ long long cnt_times(unsigned long long c, float m, float scale) {
  const uint32_t b = __float_as_uint(m);
  const int e = static_cast<int>((b >> 23) & 0xffu);
  if (e == 0 || c == 0) return 0;  // zero, or a subnormal far below the fixed-point grid
  const unsigned long long p = c * static_cast<unsigned long long>((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 150 + (static_cast<int>((__float_as_uint(scale) >> 23) & 0xffu) - 127);
  unsigned long long v;
  if (sh >= 0) v = p << (sh < 63 ? sh : 63);
  else if (sh > -64) v = (p >> -sh) + ((p >> (-sh - 1)) & 1ull);
  else v = 0;
  return (b >> 31) ? -static_cast<long long>(v) : static_cast<long long>(v);
}

// value of reverse-view task t at key k with count h
__device__ __forceinline__ long long rv_task_value(const RvTask& t, const RevView& R, const GroupDesc& G, int64_t k,
                                                   unsigned long long h, const uint32_t* rec) {
  if (t.mode == 0) return static_cast<long long>(h);
  if (t.mode == 1) return rv_slot(R, k, t.slot);
  // hist * mean * scale, one exact rounding per key
  return cnt_times(h, __uint_as_float(rec[t.mu_word]), t.scale);
}

// the reverse-view tasks too wide for a block's shared table: straight into
// their global outputs
__global__ void k_rv_tasks(const RvTask* tasks, const TaskRanges rg, const __grid_constant__ RootParams p) {
  const int r = blockIdx.y;
  const int t0 = rg.begin[r], t1 = rg.begin[r + 1];
  if (t0 == t1) return;
  const RevView& R = p.rv[r];
  const GroupDesc& G = p.grp[R.grp];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.K; k += gridDim.x * blockDim.x) {
    const unsigned long long h = rv_hist(R, k);
    if (h == 0) continue;
    const uint32_t* rec = G.rec + (int64_t)k * G.stride;
    for (int ti = t0; ti < t1; ++ti) {
      const RvTask& t = tasks[ti];
      if (t.soff >= 0) continue;  // served by the grouped launch
      int64_t cell = 0;
      for (int q = 0; q < t.n_gb; ++q) cell = cell * t.dom[q] + static_cast<int32_t>(rec[t.cat_word[q]]);
      add_ll(t.out + cell, rv_task_value(t, R, G, k, h, rec));
    }
  }
}

// Grouped reverse-view tasks: a block sums tasks [t0, t1) of one view over
// its key range in a shared-memory table (Zipf-hot categories then collide in
// shared memory instead of serialising global atomics) and adds the table to
// the outputs once.  Integer sums: the result does not depend on the order.
constexpr int kRvItemTasks = 64;  // tasks of one grouped launch block, staged in shared memory
__global__ void __launch_bounds__(256) k_rv_items(const RvTask* tasks, const RvItem* items,
                                                  const __grid_constant__ RootParams p) {
  extern __shared__ unsigned long long tab[];
  __shared__ RvTask ts[kRvItemTasks];
  const RvItem it = items[blockIdx.x];
  const RevView& R = p.rv[it.rv];
  const GroupDesc& G = p.grp[R.grp];
  for (int i = threadIdx.x; i < it.cells; i += blockDim.x) tab[i] = 0ull;
  for (int i = threadIdx.x; i < it.t1 - it.t0; i += blockDim.x) ts[i] = tasks[it.t0 + i];
  __syncthreads();
  for (int64_t k = it.k0 + threadIdx.x; k < it.k1; k += blockDim.x) {
    const unsigned long long h = rv_hist(R, k);
    if (h == 0) continue;
    const uint32_t* rec = G.rec + k * G.stride;
    for (int ti = 0; ti < it.t1 - it.t0; ++ti) {
      const RvTask& t = ts[ti];
      int64_t cell = 0;
      for (int q = 0; q < t.n_gb; ++q) cell = cell * t.dom[q] + static_cast<int32_t>(rec[t.cat_word[q]]);
      const long long v = rv_task_value(t, R, G, k, h, rec);
      if (v != 0) atomicAdd(&tab[t.soff + cell], static_cast<unsigned long long>(v));
    }
  }
  __syncthreads();
  for (int ti = 0; ti < it.t1 - it.t0; ++ti) {
    const RvTask& t = ts[ti];
    for (int64_t c = threadIdx.x; c < t.cells; c += blockDim.x) {
      const unsigned long long v = tab[t.soff + c];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(t.out + c), v);
    }
  }
}

cudaError_t launch_rv_items(const RvTask* tasks, const RvItem* items, int n_items, int max_cells,
                            const RootParams& p, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int sm = max_cells * 8;
  cudaError_t e = cudaFuncSetAttribute(k_rv_items, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  k_rv_items<<<n_items, 256, sm, s>>>(tasks, items, p);
  return cudaGetLastError();
}

// Category indexes: the keys of a probe group listed by one category value,
// rebuilt every run from the records (count, exclusive scan, scatter), one
// index per blockIdx.y.
__device__ __forceinline__ int cat_of(const GroupDesc& G, const CatIndex& I, int64_t k) {
  const int32_t v = static_cast<int32_t>(G.rec[k * G.stride + I.a_word]);
  return (v >= 0 && v < I.dom) ? v : -1;
}

__global__ void k_cat_hist(const CatIndex* idx, const __grid_constant__ RootParams p) {
  const CatIndex I = idx[blockIdx.y];
  const GroupDesc& G = p.grp[I.grp];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < G.K;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int v = cat_of(G, I, k);
    if (v >= 0) atomicAdd(I.cnt + v, 1u);
  }
}

// one block per index: exclusive scan of cnt into start, the total to
// cnt[dom] and start[dom]
__global__ void __launch_bounds__(1024) k_cat_scan(const CatIndex* idx) {
  const CatIndex I = idx[blockIdx.x];
  __shared__ uint32_t part[1024];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < I.dom; base += blockDim.x) {
    const int v = base + threadIdx.x;
    const uint32_t x = v < I.dom ? I.cnt[v] : 0u;
    part[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {  // inclusive Hillis-Steele scan
      const uint32_t y = threadIdx.x >= static_cast<unsigned>(o) ? part[threadIdx.x - o] : 0u;
      __syncthreads();
      part[threadIdx.x] += y;
      __syncthreads();
    }
    if (v < I.dom) I.start[v] = carry + part[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    I.start[I.dom] = carry;
    I.cnt[I.dom] = carry;
  }
}

// scatter: start[] ends as the end of each value's list
__global__ void k_cat_scatter(const CatIndex* idx, const __grid_constant__ RootParams p) {
  const CatIndex I = idx[blockIdx.y];
  const GroupDesc& G = p.grp[I.grp];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < G.K;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int v = cat_of(G, I, k);
    if (v >= 0) I.perm[atomicAdd(I.start + v, 1u)] = static_cast<int32_t>(k);
  }
}

cudaError_t launch_cat_index(const CatIndex* idx, int n_idx, int64_t max_K, const RootParams& p, cudaStream_t s) {
  if (n_idx <= 0) return cudaSuccess;
  const dim3 g(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((max_K + 255) / 256, 1024))),
               static_cast<unsigned>(n_idx));
  k_cat_hist<<<g, 256, 0, s>>>(idx, p);
  k_cat_scan<<<n_idx, 1024, 0, s>>>(idx);
  k_cat_scatter<<<g, 256, 0, s>>>(idx, p);
  return cudaGetLastError();
}

// COUNT table (a, b) read off category view V keyed by the task's group:
// T[a][b] = sum over the keys k with category a of V[k][b].  A block walks
// the positions [p0, p1) of the category index -- keys grouped by a -- with
// its threads on view cells b (coalesced row reads), summing in registers
// and adding to the table when a changes.  No counter sees more than one
// addition per block and value a.
__global__ void __launch_bounds__(256) k_cv_pairs(const CatViewTask* tasks, const CatIndex* idx,
                                                  const CvPairItem* items, const __grid_constant__ RootParams p) {
  __shared__ int32_t keys[256];
  __shared__ int32_t cats[256];
  const CvPairItem it = items[blockIdx.x];
  const CatViewTask T = tasks[it.task];
  const CatIndex I = idx[T.cat_idx];
  const CatView& C = p.cv[T.view];
  const GroupDesc& G = p.grp[C.grp];
  const int db = C.dom;
  const int64_t total = I.cnt[I.dom];
  const int64_t p1 = it.p1 < total ? it.p1 : total;
  const int b = it.b0 + static_cast<int>(threadIdx.x);
  const bool on = b < db;
  for (int64_t q0 = it.p0; q0 < p1; q0 += 256) {
    const int n = static_cast<int>(p1 - q0 < 256 ? p1 - q0 : 256);
    __syncthreads();
    if (static_cast<int>(threadIdx.x) < n) {
      const int32_t k = I.perm[q0 + threadIdx.x];
      keys[threadIdx.x] = k;
      cats[threadIdx.x] = cat_of(G, I, k);
    }
    __syncthreads();
    uint32_t acc = 0u;
    int a_cur = cats[0];
    for (int j0 = 0; j0 < n; j0 += 8) {  // eight independent loads in flight, then the sums
      uint32_t v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (on && j0 + u < n) ? __ldg(C.V + static_cast<int64_t>(keys[j0 + u]) * db + b) : 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (j0 + u >= n) break;
        const int a = cats[j0 + u];
        if (a != a_cur) {
          if (on && acc) {
            const int64_t cell =
                T.a_first ? static_cast<int64_t>(a_cur) * db + b : static_cast<int64_t>(b) * T.dom_a + a_cur;
            atomicAdd(reinterpret_cast<unsigned long long*>(T.out + cell), static_cast<unsigned long long>(acc));
          }
          acc = 0u;
          a_cur = a;
        }
        acc += v[u];
      }
    }
    if (on && acc) {
      const int64_t cell = T.a_first ? static_cast<int64_t>(a_cur) * db + b : static_cast<int64_t>(b) * T.dom_a + a_cur;
      atomicAdd(reinterpret_cast<unsigned long long*>(T.out + cell), static_cast<unsigned long long>(acc));
    }
  }
}

cudaError_t launch_cv_pairs(const CatViewTask* tasks, const CatIndex* idx, const CvPairItem* items, int n_items,
                            const RootParams& p, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_cv_pairs<<<n_items, 256, 0, s>>>(tasks, idx, items, p);
  return cudaGetLastError();
}

// SUM of a keying-group mean grouped by b, read off a category view: one block
// per (view, up to kCvMeanTasks of its mean tasks, range of keys, range of
// cells b); each thread takes one cell b and walks the keys, reading the
// count once for all the tasks and adding count x mean for each as one exact
// integer rounding (cnt_times); one addition per (block, task, b) at the end.
__global__ void __launch_bounds__(256) k_cv_means(const CatViewTask* tasks, const CvMeanItem* items,
                                                  const __grid_constant__ RootParams p) {
  __shared__ float mu[kCvMeanTasks][64];
  __shared__ float sc[kCvMeanTasks];
  const CvMeanItem it = items[blockIdx.x];
  const CatView& C = p.cv[it.view];
  const GroupDesc& G = p.grp[C.grp];
  const int db = C.dom;
  const int nt = it.t1 - it.t0;
  const int b = it.b0 + static_cast<int>(threadIdx.x);
  const bool on = b < db;
  if (static_cast<int>(threadIdx.x) < nt) sc[threadIdx.x] = tasks[it.t0 + threadIdx.x].scale;
  long long acc[kCvMeanTasks];
#pragma unroll
  for (int t = 0; t < kCvMeanTasks; ++t) acc[t] = 0;
  for (int64_t k0 = it.k0; k0 < it.k1; k0 += 64) {
    const int n = static_cast<int>(it.k1 - k0 < 64 ? it.k1 - k0 : 64);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * 64; e += blockDim.x) {
      const int t = e / 64, j = e % 64;
      if (j < n) mu[t][j] = __uint_as_float(G.rec[(k0 + j) * G.stride + tasks[it.t0 + t].mu_word]);
    }
    __syncthreads();
    if (!on) continue;
    for (int j0 = 0; j0 < n; j0 += 8) {  // eight independent loads in flight, then the products
      uint32_t cv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) cv[u] = j0 + u < n ? __ldg(C.V + (k0 + j0 + u) * db + b) : 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t c = cv[u];
        if (c == 0u) continue;
#pragma unroll
        for (int t = 0; t < kCvMeanTasks; ++t)
          if (t < nt) acc[t] += cnt_times(c, mu[t][j0 + u], sc[t]);
      }
    }
  }
  if (!on) return;
#pragma unroll
  for (int t = 0; t < kCvMeanTasks; ++t)
    if (t < nt && acc[t] != 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(tasks[it.t0 + t].out + b), static_cast<unsigned long long>(acc[t]));
}

cudaError_t launch_cv_means(const CatViewTask* tasks, const CvMeanItem* items, int n_items, const RootParams& p,
                            cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_cv_means<<<n_items, 256, 0, s>>>(tasks, items, p);
  return cudaGetLastError();
}

// COUNT tables read off category views: one pass over each view's cells,
// every table of the view updated from the same cell (the view read once)
__global__ void k_cv_tasks(const CatViewTask* tasks, const TaskRanges rg, const __grid_constant__ RootParams p) {
  const int v = blockIdx.y;
  const int t0 = rg.begin[v], t1 = rg.begin[v + 1];
  if (t0 == t1) return;
  const CatView& C = p.cv[v];
  const GroupDesc& G = p.grp[C.grp];
  const int64_t n = static_cast<int64_t>(G.K) * C.dom;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const long long val = static_cast<long long>(C.V[i]);
    if (val == 0) continue;
    const int64_t k = i / C.dom;
    const int b = static_cast<int>(i - k * C.dom);
    const uint32_t* rec = G.rec + k * G.stride;
    for (int t = t0; t < t1; ++t) {
      const CatViewTask& T = tasks[t];
      if (T.mode == 1) {  // count x mean: one exact rounding per cell
        add_ll(T.out + b, cnt_times(static_cast<unsigned long long>(val), __uint_as_float(rec[T.mu_word]), T.scale));
        continue;
      }
      const int a = static_cast<int32_t>(rec[T.a_word]);
      add_ll(T.out + (T.a_first ? static_cast<int64_t>(a) * C.dom + b : static_cast<int64_t>(b) * T.dom_a + a),
             val);
    }
  }
}

cudaError_t launch_cv_tasks(const CatViewTask* tasks, const TaskRanges& rg, const RootParams& p, int64_t max_cells,
                            cudaStream_t s) {
  if (rg.n_views <= 0) return cudaSuccess;
  const int64_t gb = (max_cells + 255) / 256;
  dim3 grid((unsigned)(gb < 1024 ? (gb < 1 ? 1 : gb) : 1024), (unsigned)rg.n_views);
  k_cv_tasks<<<grid, 256, 0, s>>>(tasks, rg, p);
  return cudaGetLastError();
}

// pair p of a group block: (i, j), -1 <= i <= j < n, not both -1
__device__ __forceinline__ void gg_pair(int p, int n, int& i, int& j) {
  i = -1;
  int row = n;  // pairs with first index i: n - i (i = -1 contributes n: (-1, 0..n-1))
  while (p >= row) {
    p -= row;
    ++i;
    row = n - i;
  }
  j = (i < 0 ? 0 : i) + p;
}

// Key-level sums: one warp per range of the keys.  For every key the warp
// stages the key's values in shared memory -- an integer (a count, or a
// reverse view's fixed-point slot) as two floats hi + lo (equal to it within
// 2^-48), the group's means as the FP32 values they are -- then lane l forms
// the products of its pairs l, l + 32, .. in compensated FP32 (the rounding
// error of each product recovered with an FMA) and adds them to a two-float
// (TwoSum) accumulator: each key's term carries a relative error near 2^-48,
// so a few heavy keys (Zipf-hot) cannot dominate the error.  Partials go out
// in FP64 and are summed in a fixed order.
constexpr int kGgLane = 4;
constexpr int kKeyVals = 3 * kMaxZ + 4;  // staged values of one key

__device__ __forceinline__ void ks_two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}
// an int64 as hi + lo (two floats), times a power-of-two scale
__device__ __forceinline__ void ks_split(long long v, float scale, float& hi, float& lo) {
  const float h = __ll2float_rn(v);
  hi = h * scale;
  lo = __ll2float_rn(v - __float2ll_rn(h)) * scale;
}
// acc += (ah + al) * b with the product's rounding error kept (b exact)
__device__ __forceinline__ void ks_mad(float& acc_hi, float& acc_lo, float ah, float al, float b) {
  const float p = ah * b;
  const float e = fmaf(ah, b, -p);
  ks_two_sum(acc_hi, acc_lo, p);
  acc_lo += fmaf(al, b, e);
}

__global__ void k_group_gram_part(const GroupGram* gg, int n_parts, const __grid_constant__ RootParams p,
                                  double* part) {
  __shared__ float vals[8][kKeyVals];  // per warp: [count hi, count lo, means]
  const GroupGram g = gg[blockIdx.y];
  const GroupDesc& G = p.grp[g.grp];
  const RevView& RV = p.rv[g.rv];
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  float* sv = vals[wv];
  const int64_t part_id = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wv;
  const int64_t k0 = part_id * G.K / n_parts, k1 = (part_id + 1) * G.K / n_parts;
  for (int q0 = 0; q0 < g.npair; q0 += 32 * kGgLane) {
    int pi[kGgLane], pj[kGgLane];
    float hi[kGgLane], lo[kGgLane];
#pragma unroll
    for (int u = 0; u < kGgLane; ++u) {
      const int q = q0 + lane + 32 * u;
      pi[u] = -1;
      pj[u] = 0;
      if (q < g.npair) gg_pair(q, g.n, pi[u], pj[u]);
      hi[u] = lo[u] = 0.f;
    }
    for (int64_t k = k0; k < k1; ++k) {
      const uint32_t* rec = G.rec + k * G.stride + g.mu_word;
      if (lane == 0) ks_split(static_cast<long long>(rv_hist(RV, k)), 1.f, sv[0], sv[1]);
      for (int i = lane; i < g.n; i += 32) sv[2 + i] = __uint_as_float(rec[i]);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kGgLane; ++u) {
        // m_i m_j exactly as qh + ql, then (count) x (qh + ql)
        const float mj = sv[2 + pj[u]];
        const float mi = pi[u] < 0 ? 1.f : sv[2 + pi[u]];
        const float qh = mi * mj, ql = fmaf(mi, mj, -qh);
        ks_mad(hi[u], lo[u], sv[0], sv[1], qh);
        lo[u] = fmaf(sv[0], ql, lo[u]);
      }
      __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < kGgLane; ++u) {
      const int q = q0 + lane + 32 * u;
      if (q < g.npair) part[static_cast<int64_t>(g.part_off + q) * n_parts + part_id] = (double)hi[u] + (double)lo[u];
    }
  }
}

// the partials of each pair summed in a fixed order (one warp per pair); the
// block replaces the row-level Gram entries
__global__ void k_group_gram_fin(const GroupGram* gg, int n_parts, const double* part, double* G, int m) {
  const GroupGram g = gg[blockIdx.y];
  const int lane = threadIdx.x & 31;
  for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < g.npair; q += gridDim.x * (blockDim.x >> 5)) {
    const double* src = part + static_cast<int64_t>(g.part_off + q) * n_parts;
    double s = 0.0;
    for (int c = lane; c < n_parts; c += 32) s += src[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      int i, j;
      gg_pair(q, g.n, i, j);
      const int zi = i < 0 ? 0 : g.zoff + i, zj = g.zoff + j;
      G[zi * m + zj] = s;
      G[zj * m + zi] = s;
    }
  }
}

cudaError_t launch_group_gram(const GroupGram* gg, int n_gg, int n_parts, const RootParams& p, double* part,
                              double* G, cudaStream_t s) {
  if (n_gg <= 0) return cudaSuccess;
  k_group_gram_part<<<dim3(n_parts / 8, n_gg), 256, 0, s>>>(gg, n_parts, p, part);
  k_group_gram_fin<<<dim3(16, n_gg), 256, 0, s>>>(gg, n_parts, part, G, p.m);
  return cudaGetLastError();
}

// Gram entries at the key level from the reverse views (CrossGram), in the
// form of k_group_gram_part: per key the warp stages the view's slots (exact
// fixed-point integers, scaled back to FP32) and the group's means, lane l
// forms the products of its pairs and adds them to two-float accumulators
constexpr int kCgLane = 4;
__global__ void k_cross_gram_part(const CrossGram* cg, const CrossPair* pairs, int n_parts,
                                  const __grid_constant__ RootParams p, double* part) {
  __shared__ float vals[8][kKeyVals];  // per warp: [slots hi][slots lo][means]
  const CrossGram g = cg[blockIdx.y];
  const GroupDesc& G = p.grp[g.grp];
  const RevView& R = p.rv[g.rv];
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  float* sv = vals[wv];
  const int ns = R.n_slot;
  const int64_t part_id = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wv;
  const int64_t k0 = part_id * G.K / n_parts, k1 = (part_id + 1) * G.K / n_parts;
  for (int q0 = 0; q0 < g.npair; q0 += 32 * kCgLane) {
    int ps[kCgLane], pm[kCgLane];
    float hi[kCgLane], lo[kCgLane];
#pragma unroll
    for (int u = 0; u < kCgLane; ++u) {
      const int q = q0 + lane + 32 * u;
      const CrossPair cp = q < g.npair ? pairs[g.pair_off + q] : CrossPair{0, -1, 0, 0};
      ps[u] = cp.s;
      pm[u] = cp.i;
      hi[u] = lo[u] = 0.f;
    }
    for (int64_t k = k0; k < k1; ++k) {
      const uint32_t* rec = G.rec + k * G.stride + g.mu_word;
      for (int i = lane; i < ns; i += 32) ks_split(rv_slot(R, k, i), 1.0f / R.slot_scale[i], sv[i], sv[ns + i]);
      for (int i = lane; i < G.n_mu; i += 32) sv[2 * ns + i] = __uint_as_float(rec[i]);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kCgLane; ++u) {
        const float m = pm[u] < 0 ? 1.f : sv[2 * ns + pm[u]];
        ks_mad(hi[u], lo[u], sv[ps[u]], sv[ns + ps[u]], m);
      }
      __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < kCgLane; ++u) {
      const int q = q0 + lane + 32 * u;
      if (q < g.npair) part[static_cast<int64_t>(g.part_off + q) * n_parts + part_id] = (double)hi[u] + (double)lo[u];
    }
  }
}

// the partials of each pair summed in a fixed order (one warp per pair)
__global__ void k_cross_gram_fin(const CrossGram* cg, const CrossPair* pairs, int n_parts, const double* part,
                                 double* G, int m) {
  const CrossGram g = cg[blockIdx.y];
  const int lane = threadIdx.x & 31;
  for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < g.npair; q += gridDim.x * (blockDim.x >> 5)) {
    const double* src = part + static_cast<int64_t>(g.part_off + q) * n_parts;
    double s = 0.0;
    for (int c = lane; c < n_parts; c += 32) s += src[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const CrossPair cp = pairs[g.pair_off + q];
      G[cp.za * m + cp.zb] = s;
      G[cp.zb * m + cp.za] = s;
    }
  }
}

cudaError_t launch_cross_gram(const CrossGram* cg, int n_cg, const CrossPair* pairs, int n_parts,
                              const RootParams& p, double* part, double* G, cudaStream_t s) {
  if (n_cg <= 0) return cudaSuccess;
  k_cross_gram_part<<<dim3(n_parts / 8, n_cg), 256, 0, s>>>(cg, pairs, n_parts, p, part);
  k_cross_gram_fin<<<dim3(16, n_cg), 256, 0, s>>>(cg, pairs, n_parts, part, G, p.m);
  return cudaGetLastError();
}

// key-level plans: the exact fixed-point image of every mean a reverse view
// sums, once per key (the root scan then sums integers without converting
// the same value on every row)
__global__ void k_fix_means(const __grid_constant__ FixMeans f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(f.g.K) * f.n) return;
  const int64_t k = i / f.n;
  const int j = static_cast<int>(i - k * f.n);
  const float m = __uint_as_float(f.g.rec[k * f.g.stride + f.mu_word[j]]);
  f.g.fix[k * f.g.fix_stride + j] = __float2ll_rn(m * f.scale[j]);
}

cudaError_t launch_fix_means(const FixMeans& f, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(f.g.K) * f.n;
  if (n <= 0) return cudaSuccess;
  k_fix_means<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_rv_tasks(const RvTask* tasks, const TaskRanges& rg, const RootParams& p, int max_K,
                            cudaStream_t s) {
  if (rg.n_views <= 0) return cudaSuccess;
  dim3 grid((unsigned)min((max_K + 255) / 256, 512), (unsigned)rg.n_views);
  k_rv_tasks<<<grid, 256, 0, s>>>(tasks, rg, p);
  return cudaGetLastError();
}

// final placement of every aggregate: one block per item (a map and a range
// of its cells)
__global__ void k_out_map(const OutMap* maps, const OutItem* items, const double* G, int m, const long long* count,
                          long long* res_i64, double* res_f64) {
  const OutItem it = items[blockIdx.x];
  OutMap o = maps[it.map];
  o.dst += it.c0;
  o.n = it.c1 - it.c0;
  if (o.kind >= 2) o.src += it.c0;
  const int64_t t0 = threadIdx.x;
  const int64_t step = blockDim.x;
  switch (o.kind) {
    case 0:
      if (t0 == 0) res_i64[o.dst] = *count;
      break;
    case 1:
      if (t0 == 0) res_f64[o.dst] = G[o.i * m + o.j];
      break;
    case 2:
    case 4:
      for (int64_t c = t0; c < o.n; c += step) res_i64[o.dst + c] = o.src[c];
      break;
    default:
      for (int64_t c = t0; c < o.n; c += step) res_f64[o.dst + c] = (double)o.src[c] * o.inv_scale;
      break;
  }
}

cudaError_t launch_out_map(const OutMap* maps, const OutItem* items, int n_items, const double* G, int m,
                           const long long* count, long long* res_i64, double* res_f64, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_out_map<<<n_items, 256, 0, s>>>(maps, items, G, m, count, res_i64, res_f64);
  return cudaGetLastError();
}

// the results of per-root plans placed in the batch's result arrays: one block
// per aggregate, 64-bit words copied as they are
__global__ void k_copy_results(const ResultCopy* items) {
  const ResultCopy it = items[blockIdx.x];
  for (int64_t i = threadIdx.x; i < it.n; i += blockDim.x) it.dst[i] = it.src[i];
}

cudaError_t launch_copy_results(const ResultCopy* items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_copy_results<<<n_items, 256, 0, s>>>(items);
  return cudaGetLastError();
}

}  // namespace lmf
