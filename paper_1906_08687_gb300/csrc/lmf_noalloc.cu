// lmf_noalloc.cu -- lmf_gram_noalloc: the covar Gram of one relation computed
// without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or an
// allocator of its own that forbids outside allocations, code that must not
// trigger the implicit synchronisation an allocation can cause, or a process
// that has handed all device memory to another framework.  For them this entry
// point runs the plain root-scan kernel (one row per thread, FP32 register
// blocks, per-CTA FP64 partial Grams combined in a fixed order) with its
// scratch -- the per-CTA partials and counts -- in the file-scope
// array below instead of a plan arena.  The caller passes the input columns and
// the output buffer.
//
// The array (kScratchDoubles doubles, about 2.5 MB) is part of the library's
// module: every GPU that loads the library holds it until the process exits.
// All calls share it and it keeps the last call's contents, so calls that
// overlap on the GPU (different streams, or different host threads) race.
#include "lmf.h"
#include "lmf_internal.h"

#include <mutex>

namespace {

constexpr int kMaxGrid = 304;                  // CTAs: two per SM on a 152-SM GB300
constexpr int kMaxCols = 31;                   // z = [1, x_1 .. x_31] fills the 32-wide kernel
constexpr int kMP = 32;
constexpr size_t kPartDoubles = static_cast<size_t>(kMaxGrid) * kMP * kMP;
constexpr size_t kScratchDoubles = kPartDoubles + kMaxGrid + 8;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {};       // device address of g_scratch, per device

// the reason is for a reader of this file; callers get the status code
lmf_status reject(lmf_status s, const char* /*why*/) { return s; }

// G[0][0] is COUNT: the exact int64 row count, not the FP32 sum of ones
__global__ void k_put_count(double* G, const long long* count) { G[0] = static_cast<double>(*count); }

}  // namespace

extern "C" lmf_status lmf_gram_noalloc(const float* const* dev_cols, int ncols, int64_t nrows, double* dev_gram,
                                       void* cuda_stream) {
  using namespace lmf;
  if (ncols < 0 || nrows < 0 || !dev_gram || (ncols > 0 && !dev_cols))
    return reject(LMF_ERR_ARG, "null pointer or negative size");
  if (ncols > kMaxCols) return reject(LMF_ERR_ARG, "more than 31 columns exceeds the built-in scratch");
  for (int i = 0; i < ncols; ++i)
    if (!dev_cols[i] && nrows > 0) return reject(LMF_ERR_ARG, "null column pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return reject(LMF_ERR_CUDA, "no current CUDA device");
  // one-time set-up per device, with that device current: the host-side name
  // g_scratch is not a device address, so ask the runtime for the address
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)
        return reject(LMF_ERR_CUDA, "cudaGetSymbolAddress failed");
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return reject(LMF_ERR_CUDA, "device query failed");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  const int T = root_plain_tile_rows();
  const int64_t n_tiles = (nrows + T - 1) / T;
  int64_t grid = static_cast<int64_t>(sms) * 2;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;

  RootParams p{};
  p.N = nrows;
  p.n_grp = 0;
  p.n_x = ncols;
  for (int i = 0; i < ncols; ++i) p.x[i] = {dev_cols[i], 1};
  p.n_rcat = 0;
  p.n_rowcat = 0;
  p.m = ncols + 1;
  p.gram_part = scratch;                                          // every CTA overwrites its block
  p.cnt_part = reinterpret_cast<long long*>(scratch + kPartDoubles);
  p.n_rv = 0;
  p.n_direct = 0;
  p.direct = nullptr;
  p.n_om = 0;
  // the kernel reports out-of-range categories through the status word; this
  // input has no categorical column, so nothing is ever written there and
  // nothing reads it (it only has to be a valid address)
  p.status = reinterpret_cast<uint32_t*>(scratch + kPartDoubles + kMaxGrid);
  long long* count = reinterpret_cast<long long*>(scratch + kPartDoubles + kMaxGrid + 1);

  // the partials and counts are written in full by every call: nothing to clear
  const size_t smem = root_plain_smem(kMP, 0);
  if (root_plain_prepare(kMP, smem) != cudaSuccess) return reject(LMF_ERR_CUDA, "kernel attribute failed");
  if (launch_root_plain(p, kMP, static_cast<int>(grid), n_tiles, smem, s) != cudaSuccess)
    return reject(LMF_ERR_CUDA, "root-scan launch failed");
  if (launch_combine(scratch, static_cast<int>(grid), kMP, p.m, p.cnt_part, dev_gram, count, s) != cudaSuccess)
    return reject(LMF_ERR_CUDA, "combine launch failed");
  k_put_count<<<1, 1, 0, s>>>(dev_gram, count);
  if (cudaGetLastError() != cudaSuccess) return reject(LMF_ERR_CUDA, "count placement failed");
  return LMF_OK;
}
