// lmf_root_tc.cuh -- the root scan with the covar Gram (Eq. lr-sigma, Sec. 2)
// on sm_103a tensor cores; device code only, so that the plan-specialised
// kernels compiled at plan time share it.
//
// Every root row contributes w z z^T with z = [1, root features, view means]
// (w is 0 or 1: the plan uses this kernel only when every child key is unique).
// Each FP32 z_i is split into three bf16 pieces z = h + m + l (8+8+8 bits, exact
// for FP32 input).  One tile of 128 rows gives the MMA operands
//     A (M = 128): [h; m; l; 0] blocks of 32 features,   B (N = 64): [h; m],
// K = the 128 rows, so one tile costs 8 tcgen05.mma (M128 N64 K16) and yields
// the blocks hh hm / mh mm / lh lm of sum_r A B^T in tensor memory.  With
// T0 = hh + hm, T1 = mh + mm, T2 = lh + lm the Gram is T0 + T1 + T2 + T2^T up to
// the dropped l*l term (relative 2^-32).  Every tile's accumulator is drained
// into two-float registers, so FP32 accumulation spans at most 8 MMAs.
//
// Pipeline per CTA (128 threads, one row per thread):
//   row pass of tile t (views, z, grouped updates) -> wait for the MMAs of tile
//   t-1 (they read the single operand stage) -> split/pack z into the MN-major
//   operand tiles -> one thread issues tile t's MMAs into accumulator t%2 and
//   commits them to mbarrier t%2 -> warps 0..2 drain accumulator (t-1)%2.
// Every mbarrier wait is bounded; on timeout the CTA flags the status word,
// still drains and frees its tensor memory.  The row pass is a policy
// (GenericRowPass, or the plan-specialised one).
#pragma once

#include "lmf_rowpass.cuh"

namespace lmf {

constexpr int kTcRows = 128;                      // rows per tile = K of a tile's MMAs
constexpr int kTcThreads = 128;
constexpr int kZld = 36;                          // floats per staged z row (16-B aligned)
constexpr uint32_t kAStage = 128 * kTcRows * 2;   // 32 KB bf16
constexpr uint32_t kBStage = 64 * kTcRows * 2;    // 16 KB bf16
// MN-major, no swizzle: a core matrix is 8 K-rows x 16 B (8 MN elements).
// Core matrices adjacent in K are kLBO apart, adjacent in MN kSBO apart.
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = (kTcRows / 8) * 128;    // 2048
constexpr uint32_t kTmemCols = 128;               // two accumulators of 64 FP32 columns
constexpr long long kSpinLimit = 1ll << 22;

// instruction descriptor, kind::f16: D f32, A/B bf16, both MN-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                            ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on an mbarrier phase; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// FP32 -> bf16, round to nearest even (the conversion instruction), and back
__device__ __forceinline__ uint16_t f32_to_bf16(float x) {
  uint16_t r;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float(static_cast<uint32_t>(h) << 16); }

// three-way bf16 split of an FP32 value: x == h + m + l exactly (normal range)
__device__ __forceinline__ void split3(float x, uint16_t& h, uint16_t& m, uint16_t& l) {
  h = f32_to_bf16(x);
  const float r = x - bf16_to_f32(h);
  m = f32_to_bf16(r);
  l = f32_to_bf16(r - bf16_to_f32(m));
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) {
  return static_cast<uint32_t>(a) | (static_cast<uint32_t>(b) << 16);
}

// write row k's split z into the operand tiles (MN-major core-matrix layout:
// element (mn, k) at (mn/8)*SBO + (k/8)*LBO + (k%8)*16 + (mn%8)*2)
__device__ __forceinline__ void pack_row(unsigned char* sA, unsigned char* sB, const float* zrow, int k) {
  const uint32_t koff = static_cast<uint32_t>(k >> 3) * kLBO + static_cast<uint32_t>(k & 7) * 16u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v0 = *reinterpret_cast<const float4*>(zrow + 8 * q);
    const float4 v1 = *reinterpret_cast<const float4*>(zrow + 8 * q + 4);
    const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint16_t h[8], m[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(x[e], h[e], m[e], l[e]);
    const uint4 H = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
    const uint4 M = make_uint4(pack2(m[0], m[1]), pack2(m[2], m[3]), pack2(m[4], m[5]), pack2(m[6], m[7]));
    const uint4 L = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
    *reinterpret_cast<uint4*>(sA + (0 + q) * kSBO + koff) = H;
    *reinterpret_cast<uint4*>(sA + (4 + q) * kSBO + koff) = M;
    *reinterpret_cast<uint4*>(sA + (8 + q) * kSBO + koff) = L;
    *reinterpret_cast<uint4*>(sB + (0 + q) * kSBO + koff) = H;
    *reinterpret_cast<uint4*>(sB + (4 + q) * kSBO + koff) = M;
  }
}

struct TcLayout {
  uint32_t z_off, c_off, cache_off, bar_off, slot_off, cred_off, total;
};

__host__ __device__ inline TcLayout tc_layout(int n_rowcat, int cache_cells, int res_cells) {
  TcLayout L;
  L.z_off = kAStage + kBStage;
  L.c_off = L.z_off + kTcRows * kZld * 4;
  const uint32_t ncat = n_rowcat > 0 ? n_rowcat : 1;
  L.cache_off = (L.c_off + kTcRows * ncat * 4 + 15) & ~15u;
  L.bar_off = (L.cache_off + static_cast<uint32_t>(cache_cells + res_cells) * 4 + 15) & ~15u;
  L.slot_off = L.bar_off + 16;
  L.cred_off = L.slot_off + 16;
  L.total = L.cred_off + 4 * 8;
  return L;
}

template <class RowPass>
__device__ __forceinline__ void root_tc_body(const RootParams& p, int64_t n_tiles, double* part) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcLayout L = tc_layout(p.n_rowcat, p.cache_cells, p.res_cells);
  unsigned char* sA = smem;
  uint32_t* cache = reinterpret_cast<uint32_t*>(smem + L.cache_off);
  uint32_t* res_hist = cache + p.cache_cells;
  long long res_key = -1;
  unsigned char* sB = smem + kAStage;
  float* Zs = reinterpret_cast<float*>(smem + L.z_off);
  int32_t* Cs = reinterpret_cast<int32_t*>(smem + L.c_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.slot_off);
  long long* cred = reinterpret_cast<long long*>(smem + L.cred_off);
  const int ncat = p.n_rowcat > 0 ? p.n_rowcat : 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
  const uint32_t bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};

  root_cache_zero(p, cache);
  // the fourth M block of A stays zero
  for (int i = tid; i < 4 * (int)kSBO / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(sA + 12 * kSBO)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(bar[0], 1);
    mbar_init(bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  float hi[32], lo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
  long long cnt_acc = 0;
  bool ok = true;

  auto drain = [&](int buf) {
    if (warp < 3) {
      const uint32_t src = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(buf * 64);
      float r0[32], r1[32];
      tmem_ld32(src, r0);
      tmem_ld32(src + 32, r1);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        two_sum_acc(hi[j], lo[j], r0[j]);
        lo[j] += r1[j];
      }
    }
  };

  int64_t it = 0;
  // one contiguous range of tiles per CTA: on a sorted root a CTA meets few keys
  const int64_t t_end = (blockIdx.x + 1) * n_tiles / gridDim.x;
  for (int64_t tile = blockIdx.x * n_tiles / gridDim.x; tile < t_end; ++tile, ++it) {
    const int buf = static_cast<int>(it & 1);
    float* zrow = Zs + tid * kZld;
    int32_t* crow = Cs + tid * ncat;
    if (p.res_cells > 0) root_res_advance(p, tile * kTcRows, res_hist, res_key);
    cnt_acc += RowPass::template run<32>(p, tile * kTcRows + tid, zrow, kZld, crow, p.cache_cells ? cache : nullptr,
                                         res_hist, res_key);
    if (it > 0) {  // the previous tile's MMAs read the operand stage
      const int64_t pi = it - 1;
      if (!mbar_wait(bar[pi & 1], static_cast<uint32_t>((pi >> 1) & 1))) ok = false;
      tc_fence_after();
    }
    pack_row(sA, sB, zrow, tid);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t d = tmem + static_cast<uint32_t>(buf * 64);
#pragma unroll
      for (int j = 0; j < kTcRows / 16; ++j)
        umma_bf16(d, umma_desc(aBase + j * 256u, kLBO, kSBO), umma_desc(bBase + j * 256u, kLBO, kSBO), kIdesc,
                  j > 0 ? 1u : 0u);
      umma_commit(bar[buf]);
    }
    if (it > 0) drain(1 - buf);
    tc_fence_before();
    __syncthreads();
  }
  if (it > 0) {
    const int64_t pi = it - 1;
    if (!mbar_wait(bar[pi & 1], static_cast<uint32_t>((pi >> 1) & 1))) ok = false;
    tc_fence_after();
    drain(static_cast<int>(pi & 1));
  }

  __syncthreads();
  if (p.res_cells > 0) root_res_flush(p, res_hist, res_key);
  root_cache_flush(p, cache);
  if (warp < 3) {
    double* out = part + ((static_cast<int64_t>(blockIdx.x) * 3 + warp) * 32 + lane) * 32;
#pragma unroll
    for (int j = 0; j < 32; ++j) out[j] = static_cast<double>(hi[j]) + static_cast<double>(lo[j]);
  }
  long long c = cnt_acc;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cred[warp] = c;
  if (!ok) atomicOr(p.status, kStatusTimeout);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) p.cnt_part[blockIdx.x] = cred[0] + cred[1] + cred[2] + cred[3];
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace lmf
