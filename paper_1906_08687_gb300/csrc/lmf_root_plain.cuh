// lmf_root_plain.cuh -- the plain root scan (device code only, so that the
// plan-specialised kernels compiled at plan time share it).
//
// Tiles of 256 root rows; phase 1 gives every row to one thread (the row pass:
// foreign keys, view records, z, w, grouped updates) and writes z (and w*z
// when w can exceed 1) to shared memory; phase 2 accumulates the upper
// triangle of sum_r w_r z_r z_r^T in 4x4 register blocks with FP32 FMAs,
// folded every 8 rows into a two-float (TwoSum) accumulator; each CTA
// writes its FP64 partial Gram.  The row pass is a policy: GenericRowPass
// reads the plan's descriptors, a plan-specialised one has them as constants.
#pragma once

#include "lmf_rowpass.cuh"

namespace lmf {

constexpr int kPlainT = 256;

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  float s = hi + x;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

template <int MP, class RowPass>
__device__ __forceinline__ void root_plain_body(const RootParams& p, int64_t n_tiles) {
  constexpr int T = kPlainT;
  constexpr int LD = MP + 4;
  constexpr int NBK = MP / 4;
  constexpr int NB = NBK * (NBK + 1) / 2;
  constexpr int RG = NB >= 256 ? 1 : 256 / NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // z rows; w * z rows only when w can exceed 1 (else w * z == z: dead rows are zero)
  float* Zb = reinterpret_cast<float*>(smem_raw);
  float* Za = p.unit_w ? Zb : Zb + T * LD;
  int32_t* Cs = reinterpret_cast<int32_t*>(Za + T * LD);
  uint32_t* cache = reinterpret_cast<uint32_t*>(Cs + T * (p.n_rowcat > 0 ? p.n_rowcat : 1));
  uint32_t* res_hist = cache + p.cache_cells;
  long long res_key = -1;
  const int tid = threadIdx.x;
  root_cache_zero(p, cache);
  __syncthreads();
  const int gblk = tid % NB, grow = tid / NB;
  const bool active = grow < RG;
  int bi = 0, t = gblk;
  while (t >= NBK - bi) {
    t -= NBK - bi;
    ++bi;
  }
  const int bj = bi + t;
  float hi[16], lo[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) hi[q] = lo[q] = 0.f;
  long long cnt_acc = 0;

  // one contiguous range of tiles per CTA: on a sorted root a CTA meets few keys
  const int64_t t_end = (blockIdx.x + 1) * n_tiles / gridDim.x;
  for (int64_t tile = blockIdx.x * n_tiles / gridDim.x; tile < t_end; ++tile) {
    if (p.res_cells > 0) root_res_advance(p, tile * T, res_hist, res_key);
    // ---------------- phase 1: one row per thread
    {
      const int64_t row = tile * T + tid;
      float* zrow = Zb + tid * LD;
      int32_t* crow = Cs + tid * (p.n_rowcat > 0 ? p.n_rowcat : 1);
      const long long w =
          RowPass::template run<MP>(p, row, zrow, LD, crow, p.cache_cells ? cache : nullptr, res_hist, res_key);
      cnt_acc += w;
      if (!p.unit_w) {  // w * z for the left operand
        const float wf = static_cast<float>(w);
        float* arow = Za + tid * LD;
#pragma unroll
        for (int q = 0; q < MP / 4; ++q) {
          float4 v = *reinterpret_cast<const float4*>(zrow + 4 * q);
          v.x *= wf;
          v.y *= wf;
          v.z *= wf;
          v.w *= wf;
          *reinterpret_cast<float4*>(arow + 4 * q) = v;
        }
      }
    }
    __syncthreads();
    // ---------------- phase 2: Gram blocks
    if (active) {
      // FP32 sums of at most p.fold products, each folded into the two-float
      // accumulator: on a root sorted on two or more keys consecutive rows
      // repeat the same cross products, and a long FP32 chain would round
      // them the same way in every tile
      const int fold = RowPass::fold(p) > 0 ? RowPass::fold(p) : T;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.f;
      int t = 0;
      for (int r = grow; r < T; r += RG) {
        const float4 a = *reinterpret_cast<const float4*>(Za + r * LD + 4 * bi);
        const float4 b = *reinterpret_cast<const float4*>(Zb + r * LD + 4 * bj);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(av[u], bv[v], acc[u * 4 + v]);
        if (++t == fold) {
          t = 0;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            two_sum(hi[q], lo[q], acc[q]);
            acc[q] = 0.f;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) two_sum(hi[q], lo[q], acc[q]);
    }
    __syncthreads();
  }

  if (p.res_cells > 0) root_res_flush(p, res_hist, res_key);
  root_cache_flush(p, cache);
  __syncthreads();  // the reduction below reuses the start of shared memory
  // ---------------- CTA reduction of the row groups, FP64 partial out
  double* red = reinterpret_cast<double*>(smem_raw);  // [NB * 16][RG]
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) red[(gblk * 16 + q) * RG + grow] = (double)hi[q] + (double)lo[q];
  }
  __syncthreads();
  double* out = p.gram_part + (int64_t)blockIdx.x * MP * MP;
  for (int e = tid; e < NB * 16; e += blockDim.x) {
    const int b = e / 16, q = e % 16;
    int ii = 0, tt = b;
    while (tt >= NBK - ii) {
      tt -= NBK - ii;
      ++ii;
    }
    const int jj = ii + tt;
    double s = 0.0;
    for (int g = 0; g < RG; ++g) s += red[e * RG + g];
    out[(4 * ii + q / 4) * MP + 4 * jj + q % 4] = s;
  }
  // count
  __shared__ long long cred[8];
  long long c = cnt_acc;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((tid & 31) == 0) cred[tid >> 5] = c;
  __syncthreads();
  if (tid == 0) {
    long long s = 0;
    for (int wv = 0; wv < 8; ++wv) s += cred[wv];
    p.cnt_part[blockIdx.x] = s;
  }
}


}  // namespace lmf
