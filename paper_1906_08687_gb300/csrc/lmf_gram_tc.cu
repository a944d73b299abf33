// lmf_gram_tc.cu -- the tensor-core root scan (body in lmf_root_tc.cuh) with
// the generic row pass, its ordered FP64 combine, the host-side shape and the
// bounded-wait self-test.
#include "lmf_gram_tc.h"
#include "lmf_root_tc.cuh"

namespace lmf {

namespace {

// one thread waits, bounded, on a fresh mbarrier that nothing arrives at
__global__ void k_wait_selftest(uint32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(b, 0)) atomicOr(status, kStatusTimeout);
}

__global__ void __launch_bounds__(kTcThreads) k_root_tc(const __grid_constant__ RootParams p, int64_t n_tiles,
                                                         double* part) {
  root_tc_body<GenericRowPass>(p, n_tiles, part);
}

// G[i][j] = sum over CTAs of T0 + T1 + T2 + T2^T, ordered (deterministic)
__global__ void k_combine_tc(const double* part, int grid, int m, const long long* cnt_part, double* G,
                             long long* count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m * m) {
    const int i = e / m, j = e % m;
    if (i <= j) {
      double s = 0.0;
      for (int c = 0; c < grid; ++c) {
        const double* P = part + static_cast<int64_t>(c) * 3 * 1024;
        s += P[i * 32 + j] + P[1024 + i * 32 + j] + P[2048 + i * 32 + j] + P[2048 + j * 32 + i];
      }
      G[i * m + j] = s;
      G[j * m + i] = s;
    }
  }
  if (e == 0) {
    long long s = 0;
    for (int c = 0; c < grid; ++c) s += cnt_part[c];
    *count = s;
  }
}

}  // namespace

bool gram_tc_supported(int m) { return m >= 1 && m <= 32; }
size_t gram_tc_smem(int n_rowcat, int cache_cells, int res_cells) {
  return tc_layout(n_rowcat, cache_cells, res_cells).total;
}

void gram_tc_shape(int m, int64_t N, int num_sms, int /*tile_rows*/, GramTcPlan* tp) {
  tp->m = m;
  tp->n_tiles = (N + kTcRows - 1) / kTcRows;
  tp->smem = 0;
  tp->grid = 0;
  tp->num_sms = num_sms;
}

void gram_tc_alloc(GramTcPlan* tp, const std::function<size_t(size_t)>& take) {
  tp->part_off = take(static_cast<size_t>(tp->grid) * 3 * 1024 * sizeof(double));
}

cudaError_t gram_tc_configure(GramTcPlan* tp, int n_rowcat, int ctas_per_sm, int cache_cells, int res_cells) {
  const TcLayout L = tc_layout(n_rowcat, cache_cells, res_cells);
  tp->smem = L.total;
  int cps = ctas_per_sm > 0 ? ctas_per_sm : (L.total <= 72 * 1024 ? 3 : (L.total <= 110 * 1024 ? 2 : 1));
  cps = cps > 4 ? 4 : cps;  // four CTAs of 128 tensor-memory columns fill an SM's 512
  int64_t g = static_cast<int64_t>(tp->num_sms) * cps;
  if (g > tp->n_tiles) g = tp->n_tiles;
  tp->grid = static_cast<int>(g < 1 ? 1 : g);
  return cudaFuncSetAttribute(k_root_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L.total));
}

void gram_tc_finish(GramTcPlan* tp, RootParams& /*rp*/, char* base) { tp->part = reinterpret_cast<double*>(base + tp->part_off); }

cudaError_t gram_tc_wait_selftest(uint32_t* status, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status);
  return cudaGetLastError();
}

cudaError_t gram_tc_launch(GramTcPlan* tp, const RootParams& rp, cudaStream_t s) {
  k_root_tc<<<tp->grid, kTcThreads, tp->smem, s>>>(rp, tp->n_tiles, tp->part);
  return cudaGetLastError();
}

cudaError_t gram_tc_combine(GramTcPlan* tp, const RootParams& rp, double* G, long long* count, cudaStream_t s) {
  const int mm = rp.m * rp.m;
  k_combine_tc<<<(mm + 127) / 128, 128, 0, s>>>(tp->part, tp->grid, rp.m, rp.cnt_part, G, count);
  return cudaGetLastError();
}

}  // namespace lmf
