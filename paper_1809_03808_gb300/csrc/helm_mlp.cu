// A small multilayer perceptron trained on the GPU: the cost model of the
// autotuner (predicted log solve time from grid features and a kernel
// variant).  The paper has no learned part; the direct solver itself is exact
// to rounding.
//
// Network: x (n_in) -> h1 = tanh(W1 x + b1) (n_h) -> h2 = tanh(W2 h1 + b2)
// (n_h) -> y = w3 . h2 + b3.  Loss: mean squared error over the batch.
// Parameters, contiguous FP32: W1 [n_h][n_in], b1 [n_h], W2 [n_h][n_h],
// b2 [n_h], w3 [n_h], b3 [1].  Every reduction over the batch runs in a
// fixed order (one thread per output, samples in order), so gradients and
// training are bit-reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "helm.h"
#include "helm_internal.h"

struct helm_mlp {
  int n_in = 0, n_h = 0;
  int64_t nparams = 0;
  float* p = nullptr;  // parameters
  float* g = nullptr;  // gradient
  float* m = nullptr;  // Adam first moment
  float* v = nullptr;  // Adam second moment
  int64_t step = 0;
  // activations of the last forward pass: h1, h2 [batch][n_h], y, dy [batch], dA2, dA1 [batch][n_h]
  float* act = nullptr;
  int64_t cap = 0;  // batch capacity of `act`
  float* loss = nullptr;
};

namespace {

using helm::dfree;
using helm::dmalloc;

struct Layout {
  int64_t W1, b1, W2, b2, w3, b3, n;
};
Layout layout(int n_in, int n_h) {
  Layout L;
  L.W1 = 0;
  L.b1 = L.W1 + (int64_t)n_h * n_in;
  L.W2 = L.b1 + n_h;
  L.b2 = L.W2 + (int64_t)n_h * n_h;
  L.w3 = L.b2 + n_h;
  L.b3 = L.w3 + n_h;
  L.n = L.b3 + 1;
  return L;
}

// H[s][o] = tanh(sum_i W[o][i] X[s][i] + b[o]); thread per (s, o)
__global__ void k_dense_tanh(const float* __restrict__ W, const float* __restrict__ b, const float* __restrict__ X,
                             float* __restrict__ H, int n_in, int n_out, int64_t B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n_out) return;
  const int64_t s = t / n_out;
  const int o = (int)(t - s * n_out);
  float acc = b[o];
  for (int i = 0; i < n_in; ++i) acc = fmaf(W[(int64_t)o * n_in + i], X[s * n_in + i], acc);
  H[t] = tanhf(acc);
}

// y[s] = w3 . h2[s] + b3
__global__ void k_dense_out(const float* __restrict__ w3, const float* __restrict__ b3, const float* __restrict__ H,
                            float* __restrict__ y, int n_h, int64_t B) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  float acc = b3[0];
  for (int k = 0; k < n_h; ++k) acc = fmaf(w3[k], H[s * n_h + k], acc);
  y[s] = acc;
}

// dy[s] = 2 (y - t) / B; dA2[s][k] = dy[s] w3[k] (1 - h2^2)
__global__ void k_delta_out(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ w3,
                            const float* __restrict__ H2, float* __restrict__ dy, float* __restrict__ dA2, int n_h,
                            int64_t B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * n_h) return;
  const int64_t s = i / n_h;
  const int k = (int)(i - s * n_h);
  const float d = 2.0f * (y[s] - t[s]) / (float)B;
  if (k == 0) dy[s] = d;
  const float h = H2[i];
  dA2[i] = d * w3[k] * (1.0f - h * h);
}

// dA1[s][i] = (sum_o W2[o][i] dA2[s][o]) (1 - h1^2)
__global__ void k_delta_hidden(const float* __restrict__ W2, const float* __restrict__ dA2, const float* __restrict__ H1,
                               float* __restrict__ dA1, int n_h, int64_t B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n_h) return;
  const int64_t s = t / n_h;
  const int i = (int)(t - s * n_h);
  float acc = 0.f;
  for (int o = 0; o < n_h; ++o) acc = fmaf(W2[(int64_t)o * n_h + i], dA2[s * n_h + o], acc);
  const float h = H1[t];
  dA1[t] = acc * (1.0f - h * h);
}

// gW[o][i] = sum_s D[s][o] X[s][i] (x_cols = n_in; X == nullptr: the bias,
// sum_s D[s][o]).  Thread per (o, i), samples in order.
__global__ void k_weight_grad(const float* __restrict__ D, const float* __restrict__ X, float* __restrict__ gW,
                              int n_out, int n_x, int64_t B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int cols = X ? n_x : 1;
  if (t >= (int64_t)n_out * cols) return;
  const int o = (int)(t / cols), i = (int)(t - (int64_t)o * cols);
  float acc = 0.f;
  for (int64_t s = 0; s < B; ++s) acc = fmaf(D[s * n_out + o], X ? X[s * n_x + i] : 1.0f, acc);
  gW[t] = acc;
}

// loss = mean (y - t)^2, one block, fixed order
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ loss, int64_t B) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int64_t s = threadIdx.x; s < B; s += blockDim.x) {
    const float d = y[s] - t[s];
    acc = fmaf(d, d, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = sh[0] / (float)B;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int ensure_batch(helm_mlp* m, int64_t B) {
  if (B <= m->cap) return HELM_OK;
  dfree(m->act);
  m->act = nullptr;
  m->cap = 0;
  if (dmalloc((void**)&m->act, (size_t)B * (4 * m->n_h + 2) * sizeof(float)) != cudaSuccess) return HELM_ENOMEM;
  m->cap = B;
  return HELM_OK;
}

struct Act {
  float *h1, *h2, *y, *dy, *dA2, *dA1;
};
Act acts(helm_mlp* m) {
  Act a;
  const int64_t B = m->cap;
  a.h1 = m->act;
  a.h2 = a.h1 + B * m->n_h;
  a.dA2 = a.h2 + B * m->n_h;
  a.dA1 = a.dA2 + B * m->n_h;
  a.y = a.dA1 + B * m->n_h;
  a.dy = a.y + B;
  return a;
}

cudaError_t forward(helm_mlp* m, const float* x, int64_t B, float* y) {
  const Layout L = layout(m->n_in, m->n_h);
  const Act a = acts(m);
  const int bs = 128;
  k_dense_tanh<<<blocks(B * m->n_h, bs), bs>>>(m->p + L.W1, m->p + L.b1, x, a.h1, m->n_in, m->n_h, B);
  k_dense_tanh<<<blocks(B * m->n_h, bs), bs>>>(m->p + L.W2, m->p + L.b2, a.h1, a.h2, m->n_h, m->n_h, B);
  k_dense_out<<<blocks(B, bs), bs>>>(m->p + L.w3, m->p + L.b3, a.h2, y ? y : a.y, m->n_h, B);
  return cudaGetLastError();
}

// forward + backward: m->g = dLoss/dparams, m->loss = Loss
cudaError_t gradient(helm_mlp* m, const float* x, const float* t, int64_t B) {
  cudaError_t e = forward(m, x, B, nullptr);
  if (e != cudaSuccess) return e;
  const Layout L = layout(m->n_in, m->n_h);
  const Act a = acts(m);
  const int bs = 128, nh = m->n_h;
  k_loss<<<1, 256>>>(a.y, t, m->loss, B);
  k_delta_out<<<blocks(B * nh, bs), bs>>>(a.y, t, m->p + L.w3, a.h2, a.dy, a.dA2, nh, B);
  k_weight_grad<<<blocks(nh, bs), bs>>>(a.dy, a.h2, m->g + L.w3, 1, nh, B);        // w3
  k_weight_grad<<<1, 32>>>(a.dy, nullptr, m->g + L.b3, 1, 1, B);                    // b3
  k_delta_hidden<<<blocks(B * nh, bs), bs>>>(m->p + L.W2, a.dA2, a.h1, a.dA1, nh, B);
  k_weight_grad<<<blocks((int64_t)nh * nh, bs), bs>>>(a.dA2, a.h1, m->g + L.W2, nh, nh, B);  // W2
  k_weight_grad<<<blocks(nh, bs), bs>>>(a.dA2, nullptr, m->g + L.b2, nh, 1, B);            // b2
  k_weight_grad<<<blocks((int64_t)nh * m->n_in, bs), bs>>>(a.dA1, x, m->g + L.W1, nh, m->n_in, B);  // W1
  k_weight_grad<<<blocks(nh, bs), bs>>>(a.dA1, nullptr, m->g + L.b1, nh, 1, B);                     // b1
  return cudaGetLastError();
}

// splitmix64 of (seed, i) -> uniform [-1, 1)
float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

}  // namespace

extern "C" {

int helm_mlp_create(helm_mlp_t* out, int n_in, int n_hidden, uint64_t seed) {
  if (!out) return HELM_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_in > 256 || n_hidden < 1 || n_hidden > 256) return HELM_EINVAL;
  helm_mlp* m = new (std::nothrow) helm_mlp();
  if (!m) return HELM_ENOMEM;
  m->n_in = n_in;
  m->n_h = n_hidden;
  const Layout L = layout(n_in, n_hidden);
  m->nparams = L.n;
  const size_t b = (size_t)L.n * sizeof(float);
  if (dmalloc((void**)&m->p, b) != cudaSuccess || dmalloc((void**)&m->g, b) != cudaSuccess ||
      dmalloc((void**)&m->m, b) != cudaSuccess || dmalloc((void**)&m->v, b) != cudaSuccess ||
      dmalloc((void**)&m->loss, sizeof(float)) != cudaSuccess) {
    helm_mlp_destroy(m);
    return HELM_ENOMEM;
  }
  // scaled uniform initialisation (1/sqrt(fan-in)), biases zero
  std::vector<float> h(L.n, 0.f);
  for (int64_t i = 0; i < L.b1; ++i) h[i] = hash_uniform(seed, i) / std::sqrt((float)n_in);
  for (int64_t i = L.W2; i < L.b2; ++i) h[i] = hash_uniform(seed, i) / std::sqrt((float)n_hidden);
  for (int64_t i = L.w3; i < L.b3; ++i) h[i] = hash_uniform(seed, i) / std::sqrt((float)n_hidden);
  if (cudaMemcpy(m->p, h.data(), b, cudaMemcpyHostToDevice) != cudaSuccess || cudaMemset(m->m, 0, b) != cudaSuccess ||
      cudaMemset(m->v, 0, b) != cudaSuccess) {
    helm_mlp_destroy(m);
    return HELM_ECUDA;
  }
  *out = m;
  return HELM_OK;
}

int helm_mlp_num_params(helm_mlp_t m) { return m ? (int)m->nparams : HELM_EINVAL; }

int helm_mlp_get_params(helm_mlp_t m, float* host, int n) {
  if (!m || !host || n != m->nparams) return HELM_EINVAL;
  return cudaMemcpy(host, m->p, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

int helm_mlp_set_params(helm_mlp_t m, const float* host, int n) {
  if (!m || !host || n != m->nparams) return HELM_EINVAL;
  m->step = 0;
  const size_t b = (size_t)n * sizeof(float);
  if (cudaMemcpy(m->p, host, b, cudaMemcpyHostToDevice) != cudaSuccess || cudaMemset(m->m, 0, b) != cudaSuccess ||
      cudaMemset(m->v, 0, b) != cudaSuccess)
    return HELM_ECUDA;
  return HELM_OK;
}

int helm_mlp_forward(helm_mlp_t m, const float* x, int64_t batch, float* y) {
  if (!m || !x || !y || batch < 1) return HELM_EINVAL;
  if (int rc = ensure_batch(m, batch)) return rc;
  if (forward(m, x, batch, y) != cudaSuccess) return HELM_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

int helm_mlp_gradient(helm_mlp_t m, const float* x, const float* t, int64_t batch, float* grad, float* loss) {
  if (!m || !x || !t || !grad || batch < 1) return HELM_EINVAL;
  if (int rc = ensure_batch(m, batch)) return rc;
  if (gradient(m, x, t, batch) != cudaSuccess) return HELM_ECUDA;
  if (cudaMemcpy(grad, m->g, m->nparams * sizeof(float), cudaMemcpyDeviceToDevice) != cudaSuccess) return HELM_ECUDA;
  if (loss && cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice) != cudaSuccess) return HELM_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

int helm_mlp_train(helm_mlp_t m, const float* x, const float* t, int64_t batch, int steps, float lr,
                   float* final_loss) {
  if (!m || !x || !t || batch < 1 || steps < 0 || !(lr > 0)) return HELM_EINVAL;
  if (int rc = ensure_batch(m, batch)) return rc;
  for (int s = 0; s < steps; ++s) {
    if (gradient(m, x, t, batch) != cudaSuccess) return HELM_ECUDA;
    ++m->step;
    const float c1 = 1.f - std::pow(0.9f, (float)m->step), c2 = 1.f - std::pow(0.999f, (float)m->step);
    k_adam<<<blocks(m->nparams, 256), 256>>>(m->p, m->g, m->m, m->v, m->nparams, lr, c1, c2);
  }
  if (final_loss) {
    // loss of the trained parameters
    if (gradient(m, x, t, batch) != cudaSuccess) return HELM_ECUDA;
    if (cudaMemcpy(final_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return HELM_ECUDA;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? HELM_OK : HELM_ECUDA;
}

int helm_mlp_destroy(helm_mlp_t m) {
  if (!m) return HELM_OK;
  dfree(m->p);
  dfree(m->g);
  dfree(m->m);
  dfree(m->v);
  dfree(m->act);
  dfree(m->loss);
  delete m;
  return HELM_OK;
}

}  // extern "C"
