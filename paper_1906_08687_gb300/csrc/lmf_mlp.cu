// lmf_mlp.cu -- the learned cost model of the planner: an FP32 multilayer
// perceptron  x -> ReLU(W1 x + b1) -> ReLU(W2 h1 + b2) -> w3 . h2 + b3  that
// predicts the (normalised) log run time of a candidate plan from the plan's
// features, trained with mean squared error and Adam.  Forward, backward and
// the optimiser step are hand-written kernels; every reduction runs in a fixed
// order, so training is deterministic.
//
// The paper chooses roots with a fixed rule (Sec. 3.3); the model is an
// addition of this engine that chooses among candidate plans, with the rule
// kept as the fallback (lmf_plan_learned without a model).
#include "lmf.h"
#include "lmf_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

struct lmf_mlp {
  int device = 0;
  int in = 0, hid = 0;
  int64_t n_params = 0;
  float* params = nullptr;   // W1[in][hid] b1[hid] W2[hid][hid] b2[hid] w3[hid] b3[1]
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int64_t step = 0;
  // activations for a batch of up to cap samples
  int cap = 0;
  float *xn = nullptr, *h1 = nullptr, *h2 = nullptr, *yh = nullptr, *dy = nullptr, *dh1 = nullptr, *dh2 = nullptr;
  float* loss = nullptr;
  std::vector<float> mean, stdv;
  float y_mean = 0.f, y_std = 1.f;
  float *d_mean = nullptr, *d_std = nullptr;
};

namespace {

// ---------------------------------------------------------------------------
// kernels

// (x - mean) / std per feature
__global__ void k_normalise(const float* x, int B, int K, const float* mean, const float* stdv, float* xn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * K) return;
  const int k = i % K;
  xn[i] = (x[i] - mean[k]) / stdv[k];
}

// Y[b][n] = act(sum_k X[b][k] W[k][n] + bias[n])
__global__ void k_linear_fwd(const float* X, int B, int K, const float* W, const float* bias, int N, float* Y,
                             int relu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  const int b = i / N, n = i % N;
  float s = bias[n];
  for (int k = 0; k < K; ++k) s = fmaf(X[b * K + k], W[k * N + n], s);
  Y[i] = relu ? fmaxf(s, 0.f) : s;
}

// loss = mean (yhat - y)^2 ; dy = 2 (yhat - y) / B  (one block, fixed order)
__global__ void k_mse(const float* yhat, const float* y, int B, float* dy, float* loss) {
  __shared__ float part[256];
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float e = yhat[b] - y[b];
    dy[b] = 2.f * e / B;
    s += e * e;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < blockDim.x; ++i) t += part[i];
    *loss = t / B;
  }
}

// gradient of a layer Y = act(X W + b) given dY; mask by Y > 0 when relu
// dW[k][n] = sum_b X[b][k] g[b][n],  db[n] = sum_b g[b][n]
__global__ void k_linear_wgrad(const float* X, int B, int K, const float* Y, const float* dY, int N, int relu,
                               float* dW, float* db) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K * N) {
    const int k = i / N, n = i % N;
    float s = 0.f;
    for (int b = 0; b < B; ++b) {
      const float g = (relu && Y[b * N + n] <= 0.f) ? 0.f : dY[b * N + n];
      s = fmaf(X[b * K + k], g, s);
    }
    dW[i] = s;
  } else if (i < K * N + N) {
    const int n = i - K * N;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += (relu && Y[b * N + n] <= 0.f) ? 0.f : dY[b * N + n];
    db[n] = s;
  }
}

// dX[b][k] = sum_n g[b][n] W[k][n]
__global__ void k_linear_xgrad(const float* Y, const float* dY, int B, int N, int relu, const float* W, int K,
                               float* dX) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * K) return;
  const int b = i / K, k = i % K;
  float s = 0.f;
  for (int n = 0; n < N; ++n) {
    const float g = (relu && Y[b * N + n] <= 0.f) ? 0.f : dY[b * N + n];
    s = fmaf(g, W[k * N + n], s);
  }
  dX[i] = s;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

__global__ void k_affine(const float* y, int B, float scale, float shift, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) out[i] = y[i] * scale + shift;
}

inline int nb(int64_t n) { return (int)((n + 255) / 256); }

// activation buffers for batches of up to B rows; on failure every buffer is
// freed and nulled and the capacity is 0, so a later call starts clean
lmf_status ensure_cap(lmf_mlp* m, int B) {
  if (B <= m->cap) return LMF_OK;
  float** bufs[7] = {&m->xn, &m->h1, &m->h2, &m->yh, &m->dy, &m->dh1, &m->dh2};
  const size_t b = (size_t)B;
  const size_t bytes[7] = {b * m->in * 4, b * m->hid * 4, b * m->hid * 4, b * 4, b * 4, b * m->hid * 4,
                           b * m->hid * 4};
  for (float** p : bufs) {
    cudaFree(*p);
    *p = nullptr;
  }
  m->cap = 0;
  for (int i = 0; i < 7; ++i)
    if (cudaMalloc(bufs[i], bytes[i]) != cudaSuccess) {
      for (float** p : bufs) {
        cudaFree(*p);
        *p = nullptr;
      }
      return LMF_ERR_OOM;
    }
  m->cap = B;
  return LMF_OK;
}

struct Views {
  float *W1, *b1, *W2, *b2, *w3, *b3;
};
Views views(lmf_mlp* m, float* base) {
  Views v;
  v.W1 = base;
  v.b1 = v.W1 + (int64_t)m->in * m->hid;
  v.W2 = v.b1 + m->hid;
  v.b2 = v.W2 + (int64_t)m->hid * m->hid;
  v.w3 = v.b2 + m->hid;
  v.b3 = v.w3 + m->hid;
  return v;
}

// forward on normalised inputs; leaves activations and yh (normalised target units)
void forward(lmf_mlp* m, const float* x, int B) {
  const Views P = views(m, m->params);
  k_normalise<<<nb((int64_t)B * m->in), 256>>>(x, B, m->in, m->d_mean, m->d_std, m->xn);
  k_linear_fwd<<<nb((int64_t)B * m->hid), 256>>>(m->xn, B, m->in, P.W1, P.b1, m->hid, m->h1, 1);
  k_linear_fwd<<<nb((int64_t)B * m->hid), 256>>>(m->h1, B, m->hid, P.W2, P.b2, m->hid, m->h2, 1);
  k_linear_fwd<<<nb(B), 256>>>(m->h2, B, m->hid, P.w3, P.b3, 1, m->yh, 0);
}

// gradient of the mean squared error on targets y (normalised units) into m->grads
void backward(lmf_mlp* m, const float* y, int B) {
  const Views P = views(m, m->params);
  const Views G = views(m, m->grads);
  k_mse<<<1, 256>>>(m->yh, y, B, m->dy, m->loss);
  k_linear_wgrad<<<nb((int64_t)m->hid + 1), 256>>>(m->h2, B, m->hid, m->yh, m->dy, 1, 0, G.w3, G.b3);
  k_linear_xgrad<<<nb((int64_t)B * m->hid), 256>>>(m->yh, m->dy, B, 1, 0, P.w3, m->hid, m->dh2);
  k_linear_wgrad<<<nb((int64_t)m->hid * m->hid + m->hid), 256>>>(m->h1, B, m->hid, m->h2, m->dh2, m->hid, 1, G.W2,
                                                                 G.b2);
  k_linear_xgrad<<<nb((int64_t)B * m->hid), 256>>>(m->h2, m->dh2, B, m->hid, 1, P.W2, m->hid, m->dh1);
  k_linear_wgrad<<<nb((int64_t)m->in * m->hid + m->hid), 256>>>(m->xn, B, m->in, m->h1, m->dh1, m->hid, 1, G.W1,
                                                                 G.b1);
}

// splitmix64: counter-based initialisation stream
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

lmf_status lmf_mlp_create(int device, int in_dim, int hidden, uint64_t seed, lmf_mlp** out) {
  if (!out || in_dim <= 0 || hidden <= 0 || in_dim > 4096 || hidden > 4096) return LMF_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return LMF_ERR_CUDA;
  auto* m = new lmf_mlp();
  m->device = device;
  m->in = in_dim;
  m->hid = hidden;
  m->n_params = (int64_t)in_dim * hidden + hidden + (int64_t)hidden * hidden + hidden + hidden + 1;
  const size_t bytes = (size_t)m->n_params * 4;
  if (cudaMalloc(&m->params, bytes) || cudaMalloc(&m->grads, bytes) || cudaMalloc(&m->adam_m, bytes) ||
      cudaMalloc(&m->adam_v, bytes) || cudaMalloc(&m->loss, 4) || cudaMalloc(&m->d_mean, in_dim * 4) ||
      cudaMalloc(&m->d_std, in_dim * 4)) {
    lmf_mlp_destroy(m);
    return LMF_ERR_OOM;
  }
  cudaMemset(m->adam_m, 0, bytes);
  cudaMemset(m->adam_v, 0, bytes);
  cudaMemset(m->grads, 0, bytes);
  // He-uniform weights from splitmix64, zero biases
  std::vector<float> h(m->n_params, 0.f);
  uint64_t s = seed;
  auto uni = [&]() { return (float)((splitmix64(s) >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f; };
  const float a1 = std::sqrt(6.f / in_dim), a2 = std::sqrt(6.f / hidden);
  int64_t o = 0;
  for (int64_t i = 0; i < (int64_t)in_dim * hidden; ++i) h[o++] = a1 * uni();
  o += hidden;
  for (int64_t i = 0; i < (int64_t)hidden * hidden; ++i) h[o++] = a2 * uni();
  o += hidden;
  for (int i = 0; i < hidden; ++i) h[o++] = a2 * uni() * 0.5f;
  cudaMemcpy(m->params, h.data(), bytes, cudaMemcpyHostToDevice);
  m->mean.assign(in_dim, 0.f);
  m->stdv.assign(in_dim, 1.f);
  cudaMemcpy(m->d_mean, m->mean.data(), in_dim * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_std, m->stdv.data(), in_dim * 4, cudaMemcpyHostToDevice);
  if (cudaGetLastError() != cudaSuccess) {
    lmf_mlp_destroy(m);
    return LMF_ERR_CUDA;
  }
  *out = m;
  return LMF_OK;
}

lmf_status lmf_mlp_destroy(lmf_mlp* m) {
  if (!m) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  for (float* p : {m->params, m->grads, m->adam_m, m->adam_v, m->xn, m->h1, m->h2, m->yh, m->dy, m->dh1, m->dh2,
                   m->loss, m->d_mean, m->d_std})
    if (p) cudaFree(p);
  delete m;
  return LMF_OK;
}

lmf_status lmf_mlp_num_params(lmf_mlp* m, int64_t* n) {
  if (!m || !n) return LMF_ERR_ARG;
  *n = m->n_params;
  return LMF_OK;
}

lmf_status lmf_mlp_get_params(lmf_mlp* m, float* host, int64_t n) {
  if (!m || !host || n != m->n_params) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  return cudaMemcpy(host, m->params, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

lmf_status lmf_mlp_set_params(lmf_mlp* m, const float* host, int64_t n) {
  if (!m || !host || n != m->n_params) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  return cudaMemcpy(m->params, host, n * 4, cudaMemcpyHostToDevice) == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

lmf_status lmf_mlp_set_norm(lmf_mlp* m, const float* mean, const float* stdv, float y_mean, float y_std) {
  if (!m || !mean || !stdv || !(y_std > 0.f)) return LMF_ERR_ARG;
  for (int k = 0; k < m->in; ++k)
    if (!(stdv[k] > 0.f)) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  m->mean.assign(mean, mean + m->in);
  m->stdv.assign(stdv, stdv + m->in);
  m->y_mean = y_mean;
  m->y_std = y_std;
  if (cudaMemcpy(m->d_mean, mean, m->in * 4, cudaMemcpyHostToDevice) ||
      cudaMemcpy(m->d_std, stdv, m->in * 4, cudaMemcpyHostToDevice))
    return LMF_ERR_CUDA;
  return LMF_OK;
}

lmf_status lmf_mlp_forward(lmf_mlp* m, const float* x_dev, int batch, float* y_dev) {
  if (!m || !x_dev || !y_dev || batch <= 0) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  if (ensure_cap(m, batch)) return LMF_ERR_OOM;
  forward(m, x_dev, batch);
  k_affine<<<nb(batch), 256>>>(m->yh, batch, m->y_std, m->y_mean, y_dev);
  return cudaDeviceSynchronize() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

lmf_status lmf_mlp_grad(lmf_mlp* m, const float* x_dev, const float* y_dev, int batch, float* grad_dev, float* loss) {
  if (!m || !x_dev || !y_dev || batch <= 0) return LMF_ERR_ARG;
  cudaSetDevice(m->device);
  if (ensure_cap(m, batch)) return LMF_ERR_OOM;
  forward(m, x_dev, batch);
  backward(m, y_dev, batch);
  if (grad_dev && cudaMemcpy(grad_dev, m->grads, m->n_params * 4, cudaMemcpyDeviceToDevice)) return LMF_ERR_CUDA;
  if (loss && cudaMemcpy(loss, m->loss, 4, cudaMemcpyDeviceToHost)) return LMF_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

lmf_status lmf_mlp_train_step(lmf_mlp* m, const float* x_dev, const float* y_dev, int batch, float lr, float* loss) {
  lmf_status s = lmf_mlp_grad(m, x_dev, y_dev, batch, nullptr, loss);
  if (s) return s;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  k_adam<<<nb(m->n_params), 256>>>(m->params, m->grads, m->adam_m, m->adam_v, m->n_params, lr, b1, b2, 1e-8f, c1, c2);
  return cudaDeviceSynchronize() == cudaSuccess ? LMF_OK : LMF_ERR_CUDA;
}

}  // extern "C"
