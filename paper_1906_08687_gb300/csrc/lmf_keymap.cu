// lmf_keymap.cu -- dense renumbering of sparse join keys: the key index of a
// join attribute whose values are too sparse for direct addressing (built
// when the join tree is declared, Sec. 3.1; load work, outside a run, as in
// the Sec. 4 setup).
//
// Every value is replaced by its rank among the distinct values the child
// relations hold for that attribute: rank(k) = number of distinct child keys
// below k.  A bitmap over [0, largest child key] marks the child keys; an
// exclusive prefix of the per-word popcounts gives the rank of each word's
// first key, and a popcount of the bits below k inside its word the rest.
// Values no child holds (and negative values) become -1, which never joins.
// Ranks keep the order of the keys, so the renumbering is deterministic.
#include "lmf_keymap.h"

namespace lmf {
namespace {

constexpr int kMapThreads = 256;
constexpr int kWordsPerThread = 16;
constexpr int64_t kWordsPerBlock = (int64_t)kMapThreads * kWordsPerThread;

__global__ void k_keymap_bits(const int32_t* __restrict__ keys, int64_t n, uint32_t* bits, int64_t nwords) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = keys[i];
    if (k >= 0 && (int64_t)(k >> 5) < nwords) atomicOr(bits + (k >> 5), 1u << (k & 31));
  }
}

// exclusive prefix of one value per thread over a kMapThreads-thread block;
// *total receives the block's sum (every thread)
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sum[kMapThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kMapThreads / 32 ? warp_sum[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kMapThreads / 32) warp_sum[lane] = w;
  }
  __syncthreads();
  const uint32_t before = warp ? warp_sum[warp - 1] : 0u;
  *total = warp_sum[kMapThreads / 32 - 1];
  __syncthreads();  // warp_sum is reused by the next call
  return before + x - v;
}

// keys marked in the words of block b: sums[b]
__global__ void __launch_bounds__(kMapThreads) k_keymap_block_sums(const uint32_t* bits, int64_t nwords,
                                                                   uint32_t* sums) {
  const int64_t w0 = blockIdx.x * kWordsPerBlock + (int64_t)threadIdx.x * kWordsPerThread;
  uint32_t c = 0;
  for (int j = 0; j < kWordsPerThread; ++j)
    if (w0 + j < nwords) c += __popc(bits[w0 + j]);
  uint32_t total;
  block_exclusive_scan(c, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive prefix of sums[0..nb) in place (one block); sums[nb] = the total
__global__ void __launch_bounds__(kMapThreads) k_keymap_scan_sums(uint32_t* sums, int64_t nb) {
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kMapThreads) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? sums[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

// prefix[w] = keys marked in the words before w
__global__ void __launch_bounds__(kMapThreads) k_keymap_prefix(const uint32_t* bits, int64_t nwords,
                                                               const uint32_t* sums, uint32_t* prefix) {
  const int64_t w0 = blockIdx.x * kWordsPerBlock + (int64_t)threadIdx.x * kWordsPerThread;
  uint32_t c = 0;
  for (int j = 0; j < kWordsPerThread; ++j)
    if (w0 + j < nwords) c += __popc(bits[w0 + j]);
  uint32_t total;
  uint32_t run = sums[blockIdx.x] + block_exclusive_scan(c, &total);
  for (int j = 0; j < kWordsPerThread; ++j)
    if (w0 + j < nwords) {
      prefix[w0 + j] = run;
      run += __popc(bits[w0 + j]);
    }
}

__global__ void k_keymap_apply(const int32_t* __restrict__ in, int64_t n, const uint32_t* bits,
                               const uint32_t* prefix, int64_t nwords, int32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = in[i];
    int32_t r = -1;
    if (k >= 0 && (int64_t)(k >> 5) < nwords) {
      const uint32_t word = bits[k >> 5];
      const uint32_t bit = 1u << (k & 31);
      if (word & bit) r = static_cast<int32_t>(prefix[k >> 5] + __popc(word & (bit - 1u)));
    }
    out[i] = r;
  }
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 4096 ? g : 4096);
}

}  // namespace

cudaError_t keymap_renumber(const int32_t* const* cols, const int64_t* rows, int n, int n_child, int32_t max_key,
                            int32_t* const* out, int64_t* n_keys, cudaStream_t s) {
  if (n <= 0 || n_child <= 0 || n_child > n || max_key < 0) return cudaErrorInvalidValue;
  const int64_t nwords = ((int64_t)max_key >> 5) + 1;  // at most 2^26
  const int64_t nb = (nwords + kWordsPerBlock - 1) / kWordsPerBlock;
  uint32_t* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(uint32_t) * (size_t)(2 * nwords + nb + 1));
  if (e != cudaSuccess) return e;
  uint32_t* bits = buf;
  uint32_t* prefix = buf + nwords;
  uint32_t* sums = buf + 2 * nwords;
  e = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)nwords, s);
  for (int c = 0; c < n_child && e == cudaSuccess; ++c)
    if (rows[c] > 0) {
      k_keymap_bits<<<grid_for(rows[c]), 256, 0, s>>>(cols[c], rows[c], bits, nwords);
      e = cudaGetLastError();
    }
  if (e == cudaSuccess) {
    k_keymap_block_sums<<<(unsigned)nb, kMapThreads, 0, s>>>(bits, nwords, sums);
    k_keymap_scan_sums<<<1, kMapThreads, 0, s>>>(sums, nb);
    k_keymap_prefix<<<(unsigned)nb, kMapThreads, 0, s>>>(bits, nwords, sums, prefix);
    e = cudaGetLastError();
  }
  for (int c = 0; c < n && e == cudaSuccess; ++c)
    if (rows[c] > 0) {
      k_keymap_apply<<<grid_for(rows[c]), 256, 0, s>>>(cols[c], rows[c], bits, prefix, nwords, out[c]);
      e = cudaGetLastError();
    }
  uint32_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, sums + nb, sizeof(total), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e == cudaSuccess) *n_keys = total;
  return e;
}

}  // namespace lmf
