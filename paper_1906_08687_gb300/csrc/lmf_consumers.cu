// lmf_consumers.cu -- the applications that consume an aggregate batch
// (Sec. 2), on the device: ridge linear regression by batch gradient descent
// over the covar matrix, the mutual information of categorical attribute
// pairs from the count queries of Eq. mi, and the Chow-Liu tree over those
// values.  All three read results the engine already holds in device memory;
// each is one small launch (the inputs are tiny next to the batch) with every
// reduction in a fixed order, so results repeat bit for bit.
#include "lmf.h"
#include "lmf_internal.h"

#include <cmath>

namespace {

constexpr int kBgdThreads = 256;
constexpr int kBgdMaxM = 96;        // sigma up to 96 x 96 doubles (72 KB of shared memory)
constexpr int kMiThreads = 256;
constexpr int kClMaxAttrs = 64;     // Chow-Liu over up to 64 attributes (2016 pairs)
constexpr int kClThreads = 1024;

// fixed-order block sum of one double per thread (blockDim.x a power of two);
// every thread gets the total
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < static_cast<unsigned>(o)) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// Ridge regression over the covar matrix sigma ((n+1) x (n+1), row-major, the
// last row and column the label; Sec. 2, objective J and its gradient):
//   J(theta) = 1/(2|D|) t^T sigma t + lam/2 ||theta||^2, t = (theta, -1),
//   grad_k J = 1/|D| (sigma[k, :] t) + lam theta_k.
// Each iteration takes the Barzilai-Borwein step <dtheta, dtheta> / <dtheta,
// dg> (1 on the first), halved until the Armijo condition holds, and stops
// when ||g|| <= tol max(1, ||g_0||).  J is quadratic, so the decrease of a step
// s along -g is s ||g||^2 - s^2/2 g^T H g with H = sigma[:n, :n]/|D| + lam I,
// the form the Armijo test uses (the difference of two close objective values
// would lose its digits near the optimum).  One CTA runs the whole loop.
__global__ void __launch_bounds__(kBgdThreads) k_ridge_bgd(const double* sigma_g, int m, double count, double lam,
                                                           int max_iter, double tol, double* theta_out,
                                                           int* iters_out) {
  extern __shared__ double sh[];
  const int n = m - 1;
  double* S = sh;                 // [m][m]
  double* th = S + m * m;         // theta [n]
  double* g = th + n;             // gradient [n]
  double* pth = g + n;            // previous theta
  double* pg = pth + n;           // previous gradient
  double* red = pg + n;           // [kBgdThreads]
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) S[i] = sigma_g[i];
  for (int k = threadIdx.x; k < n; k += blockDim.x) th[k] = 0.0;
  __syncthreads();
  auto gradient = [&]() {  // g = (sigma[:n, :] t) / count + lam theta, t = (theta, -1)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double s = -S[k * m + n];
      for (int j = 0; j < n; ++j) s += S[k * m + j] * th[j];
      g[k] = s / count + lam * th[k];
    }
    __syncthreads();
  };
  auto dot = [&](const double* a, const double* b) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += a[k] * b[k];
    return block_sum(v, red);
  };
  auto ghg = [&]() {  // g^T H g, H = sigma[:n, :n] / count + lam I
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += S[k * m + j] * g[j];
      v += g[k] * (s / count + lam * g[k]);
    }
    return block_sum(v, red);
  };
  gradient();
  const double g0 = sqrt(dot(g, g));
  double step = 1.0;
  bool have_prev = false;
  int it = 1;
  for (; it <= max_iter; ++it) {
    const double gg = dot(g, g);
    if (sqrt(gg) <= tol * fmax(1.0, g0)) break;
    if (have_prev) {
      // dtheta = th - pth, dg = g - pg
      double a = 0.0, b = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double dt = th[k] - pth[k], dgk = g[k] - pg[k];
        a += dt * dt;
        b += dt * dgk;
      }
      const double dd = block_sum(a, red), den = block_sum(b, red);
      if (den > 0.0) step = dd / den;
    }
    const double h = ghg();
    while (-step * gg + 0.5 * step * step * h > -0.5 * step * gg) step *= 0.5;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      pth[k] = th[k];
      pg[k] = g[k];
      th[k] = th[k] - step * g[k];
    }
    have_prev = true;
    __syncthreads();
    gradient();
  }
  if (it > max_iter) it = max_iter + 1;
  for (int k = threadIdx.x; k < n; k += blockDim.x) theta_out[k] = th[k];
  if (threadIdx.x == 0) *iters_out = it - 1;
}

// Mutual information of one categorical pair per block (Sec. 2, Eq. mi):
//   MI = sum_{a, b: delta_ab > 0} delta_ab / alpha * log(alpha delta_ab / (beta_a gamma_b)),
// alpha = COUNT, beta = COUNT by X_i, gamma = COUNT by X_j, delta = COUNT by
// (X_i, X_j), row-major dom_i x dom_j.  The terms are summed per thread in cell
// order, then over the threads in a fixed tree.
__global__ void __launch_bounds__(kMiThreads) k_mutual_information(const lmf_mi_pair* pairs, long long alpha,
                                                                    double* out) {
  __shared__ double red[kMiThreads];
  const lmf_mi_pair P = pairs[blockIdx.x];
  const int64_t cells = static_cast<int64_t>(P.dom_i) * P.dom_j;
  const double A = static_cast<double>(alpha);
  double v = 0.0;
  for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
    const long long d = P.delta[c];
    if (d <= 0) continue;
    const double be = static_cast<double>(P.beta[c / P.dom_j]), ga = static_cast<double>(P.gamma[c % P.dom_j]);
    const double dd = static_cast<double>(d);
    v += dd / A * log(A * dd / (be * ga));
  }
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Chow-Liu tree (Sec. 2): the pairs in decreasing mutual information (ties:
// the pair (i, j), i < j, first in row-major order), each kept unless it closes
// a cycle -- a maximum spanning tree.  One CTA: every thread ranks its pairs by
// counting the pairs that come before them, then thread 0 walks the order with
// a union-find.
__global__ void __launch_bounds__(kClThreads) k_chow_liu(const double* mi, int n, int* edges, int* n_edges) {
  __shared__ int order[kClMaxAttrs * (kClMaxAttrs - 1) / 2];
  __shared__ int parent[kClMaxAttrs];
  const int E = n * (n - 1) / 2;
  auto pair_of = [&](int e, int* i, int* j) {  // e-th pair (i, j), i < j, in row-major order (0 <= e < E)
    int a = 0, r = e;
    while (a < n - 1 && r >= n - 1 - a) {
      r -= n - 1 - a;
      ++a;
    }
    *i = a;
    *j = a + 1 + r;
  };
  // a NaN weight ranks below every number, so the ranks form a permutation
  auto weight = [&](int i, int j) {
    const double u = mi[i * n + j];
    return isnan(u) ? -INFINITY : u;
  };
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    int i, j;
    pair_of(e, &i, &j);
    const double w = weight(i, j);
    int rank = 0, f = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q, ++f) {
        const double u = weight(p, q);
        if (u > w || (u == w && f < e)) ++rank;
      }
    order[rank] = e;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) parent[i] = i;
  __syncthreads();
  if (threadIdx.x != 0) return;
  int k = 0;
  for (int r = 0; r < E && k < n - 1; ++r) {
    int i, j;
    pair_of(order[r], &i, &j);
    int ri = i, rj = j;
    while (parent[ri] != ri) ri = parent[ri];
    while (parent[rj] != rj) rj = parent[rj];
    if (ri == rj) continue;
    parent[ri] = rj;
    edges[2 * k] = i;
    edges[2 * k + 1] = j;
    ++k;
  }
  *n_edges = k;
}

}  // namespace

extern "C" lmf_status lmf_ridge_bgd(const double* dev_sigma, int m, double count, double lam, int max_iter,
                                    double tol, double* dev_theta, int* dev_iters, void* cuda_stream) {
  if (!dev_sigma || !dev_theta || !dev_iters || m < 2 || m > kBgdMaxM || !(count > 0.0) || lam < 0.0 ||
      max_iter < 0 || !(tol >= 0.0))
    return LMF_ERR_ARG;
  const int n = m - 1;
  const size_t smem = (static_cast<size_t>(m) * m + 4 * static_cast<size_t>(n) + kBgdThreads) * sizeof(double);
  if (cudaFuncSetAttribute(k_ridge_bgd, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return LMF_ERR_CUDA;
  k_ridge_bgd<<<1, kBgdThreads, smem, static_cast<cudaStream_t>(cuda_stream)>>>(dev_sigma, m, count, lam, max_iter,
                                                                              tol, dev_theta, dev_iters);
  return cudaGetLastError() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

extern "C" lmf_status lmf_mutual_information(const lmf_mi_pair* dev_pairs, int n_pairs, int64_t alpha,
                                             double* dev_mi, void* cuda_stream) {
  if (n_pairs < 0 || (n_pairs > 0 && (!dev_pairs || !dev_mi)) || alpha <= 0) return LMF_ERR_ARG;
  if (n_pairs == 0) return LMF_OK;
  k_mutual_information<<<n_pairs, kMiThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev_pairs, alpha, dev_mi);
  return cudaGetLastError() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

extern "C" lmf_status lmf_chow_liu(const double* dev_mi, int n, int* dev_edges, int* dev_n_edges, void* cuda_stream) {
  if (!dev_mi || !dev_edges || !dev_n_edges || n < 1 || n > kClMaxAttrs) return LMF_ERR_ARG;
  k_chow_liu<<<1, kClThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(dev_mi, n, dev_edges, dev_n_edges);
  return cudaGetLastError() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}
