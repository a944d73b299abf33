// lmf_root_lean.cuh -- the key-level root scan (device code only; the plan's
// row pass is generated and compiled at plan time by lmf_jit.cu).
//
// The covar Gram of Eq. lr-sigma (Sec. 2) splits into blocks by where its two
// factors live.  Products of two root features vary from row to row and are
// summed row by row here (FP32 in 4x4 register blocks, folded into two-float
// accumulators).  Every block with a view mean m_g factors over the key of g,
// because m_g is constant on the root rows with one key:
//     sum_r z_a(r) m_{g,i}(k_g(r)) = sum_k m_{g,i}(k) R_g[k][a],
//     R_g[k][a] = sum of z_a over the root rows with k_g = k,
// i.e. the aggregate taken at the root of g (Sec. 3.3) over the directional
// view from the root towards g (Sec. 3.2).  The scan builds, per probe group,
// that reverse view -- the count and the slots its Gram blocks and grouped
// outputs need -- and leaves the products to key-level kernels
// (k_cross_gram_*, k_group_gram_*).
//
// Every value a reverse view sums is turned once per row into an exact
// fixed-point integer (a power-of-two scaling, rounded) in the row's int64
// tile row, so that every later sum is exact and order-free.  Reverse-view
// updates (RevView::mode), record [K][stride] int64, word 0 the count, word
// 1 + s slot s:
//   runs      rows sorted on the key (runs of equal keys in a warp): lane w
//             sums word w over each run and issues one reduction per run; or,
//             when the record is the first columns of the tile row, writes
//             the run's sums into the run's last row, whose thread adds the
//             whole record with one bulk reduction;
//   resident  the CTA's resident key (the first sort attribute of the root,
//             the outer loop of the trie scan of Sec. 3.5): when a warp's 32
//             rows all carry it, lane w adds the warp's sum of word w to a
//             register, added to the view once, when the key changes;
//   bulk      keys that change from row to row: the row's record (its first
//             tile columns) is added to the view by one bulk reduction
//             (cp.reduce.async.bulk ... .add.u64), which the TMA unit performs
//             in L2 without the SM issuing one reduction per word.
// The row pass is a policy (the generated JitLeanPass) that also provides the
// shared-memory layout as constants.
#pragma once

#include "lmf_root_plain.cuh"

namespace lmf {

constexpr int kLeanFoldTiles = 8;     // tiles per FP32 chain of the row Gram before the two-float fold

// round(z * 2^e) to the nearest integer (ties away from zero), exactly, with
// integer operations: z = +-m * 2^(ez - 150) with the 24-bit significand m, so
// z * 2^e = m * 2^sh, a left shift or a rounded right shift of m.  The plan's
// scales keep |z| * 2^e below 2^62.
__device__ __forceinline__ long long lean_fx(float z, int e) {
  const uint32_t b = __float_as_uint(z);
  const int ez = static_cast<int>((b >> 23) & 0xffu);
  const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
  const int sh = ez - 150 + e;
  unsigned long long v;
  if (sh >= 0) v = m << (sh < 63 ? sh : 63);
  else if (sh > -26) v = (m + (1ull << (-sh - 1))) >> -sh;
  else v = 0ull;
  if (ez == 0) v = 0ull;  // zero (and subnormals, below any scale's resolution)
  return (b >> 31) ? -static_cast<long long>(v) : static_cast<long long>(v);
}

// reduction into a reverse view: nothing in the scan reads the views, so the
// compiler may move shared-memory loads across it (no memory clobber)
__device__ __forceinline__ void lean_red_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v));
}

// sum of record word w (column col of the warp's fixed-point rows, exact
// integers) over every run of equal keys among the warp's 32 rows, one
// reduction per run; ziw: the warp's first fixed-point row (rows ld words
// apart), fk: this lane's key (-1: dead row, its row is zero); every lane of
// the warp calls this
__device__ __forceinline__ long long lean_warp_sum(const long long* ziw, int ld, int col) {
  long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // four independent chains
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    a0 += ziw[(j + 0) * ld + col];
    a1 += ziw[(j + 1) * ld + col];
    a2 += ziw[(j + 2) * ld + col];
    a3 += ziw[(j + 3) * ld + col];
  }
  return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ void lean_rv_runs(const WarpRuns& q, long long fk, const long long* ziw, int ld, int col,
                                             bool on, unsigned long long* rec0, int stride, int w) {
  if (q.heads == 1u) {  // one run over the whole warp (warp-uniform)
    const long long acc = lean_warp_sum(ziw, ld, col);
    const long long k0 = __shfl_sync(kFullWarp, fk, 0);
    if (on && k0 >= 0 && acc != 0) lean_red_u64(rec0 + k0 * stride + w, static_cast<unsigned long long>(acc));
    return;
  }
  long long acc = 0;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    acc += ziw[j * ld + col];
    if (j == 31 || ((q.heads >> (j + 1)) & 1u)) {  // row j ends a run (warp-uniform)
      const long long kj = __shfl_sync(kFullWarp, fk, j);
      if (on && kj >= 0 && acc != 0) lean_red_u64(rec0 + kj * stride + w, static_cast<unsigned long long>(acc));
      acc = 0;
    }
  }
}

// run sums of column col written in place: the sum over each run of equal
// keys replaces the column's value in the run's last row (the rows are the
// warp's own, each lane reads and writes only its column); every lane of the
// warp calls this
__device__ __forceinline__ void lean_rv_inplace(const WarpRuns& q, long long* ziw, int ld, int col, bool on) {
  if (!on) return;
  long long acc = 0;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    acc += ziw[j * ld + col];
    if (j == 31 || ((q.heads >> (j + 1)) & 1u)) {  // row j ends a run
      ziw[j * ld + col] = acc;
      acc = 0;
    }
  }
}

// the resident key's view: a warp whose 32 rows all carry the resident key adds
// its sums to the lane's register racc; any other warp takes the runs path
__device__ __forceinline__ void lean_rv_resident(const WarpRuns& q, long long fk, long long res_key,
                                                 const long long* ziw, int ld, int col, bool on, long long& racc,
                                                 unsigned long long* rec0, int stride, int w) {
  const long long k0 = __shfl_sync(kFullWarp, fk, 0);
  if (q.heads == 1u && k0 >= 0 && k0 == res_key) {  // warp-uniform
    const long long acc = lean_warp_sum(ziw, ld, col);
    if (on) racc += acc;
    return;
  }
  lean_rv_runs(q, fk, ziw, ld, col, on, rec0, stride, w);
}

// one bulk reduction of `bytes` (a multiple of 16) from this thread's staged
// record to the view record at dst (16-byte aligned)
__device__ __forceinline__ void lean_bulk_add(unsigned long long* dst, const unsigned long long* st, int bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(dst),
               "r"(static_cast<uint32_t>(__cvta_generic_to_shared(st))), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the staged records of this thread may be overwritten once its earlier bulk
// reductions have read them
__device__ __forceinline__ void lean_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void lean_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// at the start of a tile: make the key of the tile's first row resident,
// flushing the previous key's shared counters and every warp's registers;
// every thread of the CTA calls this
template <class RowPass>
__device__ __forceinline__ void lean_res_advance(const RootParams& p, int64_t row0, uint32_t* hist, long long& key,
                                                 long long* racc) {
  long long nk = -1;
  if (row0 < p.N) {
    const GroupDesc& G = p.grp[p.res_grp];
    const int32_t f = G.fk[row0];
    nk = (f >= 0 && f < G.K) ? f : -1;
  }
  if (nk == key) return;
  __syncthreads();  // the counts of earlier tiles are in
  if (p.res_cells > 0) root_res_flush(p, hist, key);
  RowPass::flush_resident(p, racc, key);
  __syncthreads();  // cleared before the next tile counts
  key = nk;
}

template <class RowPass>
__device__ __forceinline__ void root_lean_body(const RootParams& p, int64_t n_tiles) {
  constexpr int T = kLeanT;
  constexpr int MPX = RowPass::kMpx;
  constexpr int NBK = MPX / 4;
  constexpr int NB = NBK * (NBK + 1) / 2;
  constexpr int RG = NB >= 256 ? 1 : 256 / NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* Zi = reinterpret_cast<long long*>(smem_raw);
  float* Xg = reinterpret_cast<float*>(smem_raw + RowPass::kXgOff);
  float* Zf = reinterpret_cast<float*>(smem_raw + RowPass::kZfOff);
  unsigned long long* stage = reinterpret_cast<unsigned long long*>(smem_raw + RowPass::kStageOff);
  int32_t* Cs = reinterpret_cast<int32_t*>(smem_raw + RowPass::kCatOff);
  uint32_t* cache = reinterpret_cast<uint32_t*>(smem_raw + RowPass::kCacheOff);
  uint32_t* res_hist = cache + p.cache_cells;
  long long res_key = -1;
  long long racc[RowPass::kRacc];
#pragma unroll
  for (int c = 0; c < RowPass::kRacc; ++c) racc[c] = 0;
  const int tid = threadIdx.x;
  root_cache_zero(p, cache);
  __syncthreads();
  const int gblk = tid % NB, grow = tid / NB;
  const bool active = grow < RG;
  int bi = 0, tb = gblk;
  while (tb >= NBK - bi) {
    tb -= NBK - bi;
    ++bi;
  }
  const int bj = bi + tb;
  // the row Gram: FP32 chains in registers (a 4x4 block of the upper
  // triangle per thread, RG threads per block); every kLeanFoldTiles tiles the
  // chains of a block entry are summed into one two-float total held by the
  // entry's owner thread (entry e = block * 16 + q owned by thread e mod 256)
  constexpr int NE = (NB * 16 + T - 1) / T;
  float acc[16], ghi[NE], glo[NE];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
#pragma unroll
  for (int e = 0; e < NE; ++e) ghi[e] = glo[e] = 0.f;
  int fold_t = 0;
  // fold: the chains go through shared memory at the start of the tile (the
  // fixed-point tile is free between tiles once this thread's bulk
  // reductions have read it); every thread of the CTA calls this
  auto fold = [&]() {
    float* st = reinterpret_cast<float*>(smem_raw);  // [16][T]
    lean_bulk_wait_read();
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      st[q * T + tid] = active ? acc[q] : 0.f;
      acc[q] = 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int ent = tid + e * T;
      if (ent < NB * 16) {
        const int b = ent / 16, q = ent % 16;
        for (int g = 0; g < RG; ++g) two_sum(ghi[e], glo[e], st[q * T + g * NB + b]);
      }
    }
    __syncthreads();
  };
  long long cnt_acc = 0;
  const bool resident = RowPass::kResident && p.res_grp >= 0;

  // the root's columns of the next tile are loaded while this one is processed
  const int64_t t_begin = blockIdx.x * n_tiles / gridDim.x;
  const int64_t t_end = (blockIdx.x + 1) * n_tiles / gridDim.x;
  typename RowPass::Row cur, nxt;
  if (t_begin < t_end) RowPass::load(p, t_begin * T + tid, cur);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    if (tile + 1 < t_end) RowPass::load(p, (tile + 1) * T + tid, nxt);
    if (resident) lean_res_advance<RowPass>(p, tile * T, res_hist, res_key, racc);
    cnt_acc += RowPass::run(p, tile * T + tid, cur, Zi + tid * RowPass::kZiLd, Xg + tid * MPX,
                            Zf + tid * RowPass::kZfLd, Cs + tid * RowPass::kCatW, p.cache_cells ? cache : nullptr,
                            res_hist, res_key, racc, stage + tid * RowPass::kStageW);
    cur = nxt;
    __syncthreads();
    // row-level Gram of the root's features
    if (active) {
      for (int r = grow; r < T; r += RG) {
        const float4 a = *reinterpret_cast<const float4*>(Xg + r * MPX + 4 * bi);
        const float4 b = *reinterpret_cast<const float4*>(Xg + r * MPX + 4 * bj);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(av[u], bv[v], acc[u * 4 + v]);
      }
    }
    __syncthreads();
    if (++fold_t == kLeanFoldTiles) {  // products of root features vary row by row: no value repeats
      fold_t = 0;                      // along a chain, and the fold bounds its length
      fold();
    }
  }
  fold();
  if (resident) {
    if (p.res_cells > 0) root_res_flush(p, res_hist, res_key);
    RowPass::flush_resident(p, racc, res_key);
  }
  root_cache_flush(p, cache);
  lean_bulk_wait_all();
  double* out = p.gram_part + (int64_t)blockIdx.x * MPX * MPX;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int ent = tid + e * T;
    if (ent < NB * 16) {
      const int b = ent / 16, q = ent % 16;
      int ii = 0, tt = b;
      while (tt >= NBK - ii) {
        tt -= NBK - ii;
        ++ii;
      }
      const int jj = ii + tt;
      out[(4 * ii + q / 4) * MPX + 4 * jj + q % 4] = (double)ghi[e] + (double)glo[e];
    }
  }
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
