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
__device__ __forceinline__ void rp_add_ll(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
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

// grouped updates of one joining row (w != 0); cache (may be null) holds the
// CTA's counters for the hot cells of pair-count tables
__device__ __forceinline__ void root_row_grouped(const RootParams& p, int64_t row, const float* zrow,
                                                 const int32_t* crow, long long w, uint32_t* cache) {
  for (int r = 0; r < p.n_rv; ++r) {
    const RevView& R = p.rv[r];
    const int32_t fk = p.grp[R.grp].fk[row];
    atomicAdd(R.hist + fk, static_cast<unsigned long long>(w));
    long long* dst = R.R + (int64_t)fk * R.n_slot;
    for (int s = 0; s < R.n_slot; ++s) rp_add_ll(dst + s, rp_fixp(w, zrow[R.slot_z[s]], R.slot_scale[s]));
  }
  for (int d = 0; d < p.n_direct; ++d) {
    const DirectAgg& A = p.direct[d];
    const long long v = A.z < 0 ? w : rp_fixp(w, zrow[A.z], A.scale);
    if (cache && A.cache_off >= 0) {  // a pair-count table: 32-bit counter cells
      const int ha = __ldg(p.hot_lut + p.hot_lut_off[A.cat[0]] + crow[A.cat[0]]);
      const int hb = __ldg(p.hot_lut + p.hot_lut_off[A.cat[1]] + crow[A.cat[1]]);
      if (ha >= 0 && hb >= 0) {
        atomicAdd(cache + A.cache_off + ha * p.hot_h + hb, static_cast<uint32_t>(v));
        continue;
      }
    }
    int64_t cell = 0;
    for (int q = 0; q < A.n_gb; ++q) cell = cell * A.dom[q] + crow[A.cat[q]];
    rp_add_ll(A.out + cell, v);
  }
  for (int o = 0; o < p.n_om; ++o) {
    const OmegaAcc& O = p.om[o];
    const GroupDesc& G = p.grp[O.grp];
    const int32_t fk = G.fk[row];
    const long long ce = static_cast<long long>(G.rec[(int64_t)fk * G.stride + O.cnt_word]);
    atomicAdd(O.omega + fk, static_cast<unsigned long long>(w / ce));
  }
}

// the CTA's cache of 32-bit counters: zero at start, flush to the global
// int64 cells at the end
__device__ __forceinline__ void root_cache_zero(const RootParams& p, uint32_t* cache) {
  for (int i = threadIdx.x; i < p.cache_cells; i += blockDim.x) cache[i] = 0u;
}
__device__ __forceinline__ void root_cache_flush(const RootParams& p, const uint32_t* cache) {
  for (int i = threadIdx.x; i < p.cache_cells; i += blockDim.x) {
    const unsigned long long v = cache[i];
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(p.cache_dst[i]), v);
  }
}

template <int MP>
__device__ __forceinline__ long long root_row_pass(const RootParams& p, int64_t row, float* zrow,
                                                   int32_t* crow, uint32_t* cache) {
  const long long w = root_row_z<MP>(p, row, zrow, crow);
  if (w != 0) root_row_grouped(p, row, zrow, crow, w, cache);
  return w;
}

}  // namespace lmf
