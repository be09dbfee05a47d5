// Cost model of the learned tuner (include/pjds_mlp.h): training and
// inference kernels for a 15 -> 64 -> 64 -> 1 ReLU perceptron, the host
// training loop, the matrix features / candidate encoding, and the choice of
// a launch configuration (the model inside its feature range, the exhaustive
// sweep outside it).
//
// One CTA of 256 threads handles 64 samples at a time with every parameter
// and activation in shared memory (the model has 5121 parameters). W2 is kept
// twice, row-major and transposed, so that both the forward product (lanes
// over output units) and the backward product (lanes over input units) read
// shared memory without bank conflicts. Each CTA writes the gradient of its
// samples to its own slot; a second kernel adds the slots in CTA order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.h"
#include "pjds_mlp.h"
#include "pjds_tune.h"

namespace pjds {
namespace mlp {

constexpr int IN = PJDS_MLP_IN, H = PJDS_MLP_HID, SB = 64, NT = 256;
constexpr int O_W1 = 0, O_B1 = O_W1 + H * IN, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H,
              O_B3 = O_W3 + H, NP = O_B3 + 1;
constexpr int NP4 = (NP + 3) & ~3;

// shared-memory layout (floats)
constexpr int S_P = 0, S_W2T = S_P + NP4, S_X = S_W2T + H * H, S_Z1 = S_X + SB * IN, S_Z2 = S_Z1 + SB * H,
              S_OUT = S_Z2 + SB * H, S_FWD_END = S_OUT + SB;
constexpr int S_DZ2 = S_FWD_END, S_G = S_DZ2 + SB * H, S_GRAD_END = S_G + NP4;

// Forward pass of up to SB samples whose standardised inputs are rows idx[0..cnt)
// (or rows first..first+cnt when idx is NULL) of X; leaves z1, z2 and out in
// shared memory.
__device__ void forward_tile(float *sm, const float *__restrict__ P, const float *__restrict__ X,
                             const int32_t *__restrict__ idx, int64_t first, int cnt) {
  float *p = sm + S_P, *w2t = sm + S_W2T, *xs = sm + S_X, *z1 = sm + S_Z1, *z2 = sm + S_Z2, *out = sm + S_OUT;
  for (int q = threadIdx.x; q < NP; q += NT) p[q] = P[q];
  __syncthreads();
  for (int q = threadIdx.x; q < H * H; q += NT) {
    const int h = q / H, k = q % H;
    w2t[k * H + h] = p[O_W2 + q];
  }
  for (int q = threadIdx.x; q < SB * IN; q += NT) {
    const int s = q / IN, i = q % IN;
    float v = 0.0f;
    if (s < cnt) {
      const int64_t row = idx ? (int64_t)idx[s] : first + s;
      v = X[row * IN + i];
    }
    xs[q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < SB * H; q += NT) {  // z1 = x W1^T + b1
    const int s = q / H, h = q % H;
    float a = p[O_B1 + h];
    for (int i = 0; i < IN; ++i) a = fmaf(xs[s * IN + i], p[O_W1 + h * IN + i], a);
    z1[q] = a;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < SB * H; q += NT) {  // z2 = relu(z1) W2^T + b2
    const int s = q / H, h = q % H;
    float a = p[O_B2 + h];
    for (int k = 0; k < H; ++k) a = fmaf(fmaxf(z1[s * H + k], 0.0f), w2t[k * H + h], a);
    z2[q] = a;
  }
  __syncthreads();
  {  // out = relu(z2) w3 + b3: one warp per sample, lanes over units
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int s = w; s < SB; s += NT / 32) {
      float a = fmaxf(z2[s * H + l], 0.0f) * p[O_W3 + l] + fmaxf(z2[s * H + l + 32], 0.0f) * p[O_W3 + l + 32];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (l == 0) out[s] = a + p[O_B3];
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT)
    forward_kernel(const float *__restrict__ P, const float *__restrict__ X, int32_t n, float *__restrict__ out) {
  extern __shared__ float sm[];
  const int64_t first = (int64_t)blockIdx.x * SB;
  const int64_t left = n - first;
  const int cnt = left < SB ? (int)left : SB;
  forward_tile(sm, P, X, nullptr, first, cnt);
  for (int s = threadIdx.x; s < cnt; s += NT) out[first + s] = sm[S_OUT + s];
}

// Gradient of (1/n_batch) sum (out - y)^2 over this CTA's samples -> partial[blockIdx.x][NP]
__global__ void __launch_bounds__(NT)
    grad_kernel(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ Y,
                const int32_t *__restrict__ idx, int32_t n_batch, float inv_n, float *__restrict__ partial) {
  extern __shared__ float sm[];
  const int base = blockIdx.x * SB;
  const int left = n_batch - base;
  const int cnt = left < 0 ? 0 : (left < SB ? left : SB);
  forward_tile(sm, P, X, idx + base, 0, cnt);
  float *p = sm + S_P, *xs = sm + S_X, *z1 = sm + S_Z1, *z2 = sm + S_Z2, *out = sm + S_OUT;
  float *dz2 = sm + S_DZ2, *g = sm + S_G;
  // d_out (in place of out)
  for (int s = threadIdx.x; s < SB; s += NT) out[s] = s < cnt ? 2.0f * (out[s] - Y[idx[base + s]]) * inv_n : 0.0f;
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += NT) {  // dw3, db3
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a = fmaf(fmaxf(z2[s * H + k], 0.0f), out[s], a);
    g[O_W3 + k] = a;
  }
  if (threadIdx.x == 0) {
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a += out[s];
    g[O_B3] = a;
  }
  for (int q = threadIdx.x; q < SB * H; q += NT) {  // dz2
    const int s = q / H, h = q % H;
    dz2[q] = z2[q] > 0.0f ? out[s] * p[O_W3 + h] : 0.0f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < H * H; q += NT) {  // dW2[h][k] = sum_s dz2[s][h] relu(z1[s][k])
    const int h = q / H, k = q % H;
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a = fmaf(dz2[s * H + h], fmaxf(z1[s * H + k], 0.0f), a);
    g[O_W2 + q] = a;
  }
  for (int h = threadIdx.x; h < H; h += NT) {  // db2
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a += dz2[s * H + h];
    g[O_B2 + h] = a;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < SB * H; q += NT) {  // dz1 (into z2's slot): (dz2 W2) * (z1 > 0)
    const int s = q / H, k = q % H;
    float a = 0.0f;
    for (int h = 0; h < H; ++h) a = fmaf(dz2[s * H + h], p[O_W2 + h * H + k], a);
    z2[q] = z1[q] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  const float *dz1 = z2;
  for (int q = threadIdx.x; q < H * IN; q += NT) {  // dW1[h][i] = sum_s dz1[s][h] x[s][i]
    const int h = q / IN, i = q % IN;
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a = fmaf(dz1[s * H + h], xs[s * IN + i], a);
    g[O_W1 + q] = a;
  }
  for (int h = threadIdx.x; h < H; h += NT) {  // db1
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a += dz1[s * H + h];
    g[O_B1 + h] = a;
  }
  __syncthreads();
  float *dst = partial + (int64_t)blockIdx.x * NP;
  for (int q = threadIdx.x; q < NP; q += NT) dst[q] = g[q];
}

// grad[q] = sum over CTAs c = 0, 1, ... of partial[c][q]
__global__ void reduce_kernel(const float *__restrict__ partial, int32_t n_parts, float *__restrict__ grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NP) return;
  float a = 0.0f;
  for (int c = 0; c < n_parts; ++c) a += partial[(int64_t)c * NP + q];
  grad[q] = a;
}

// Adam (Kingma & Ba 2015, Algorithm 1); c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ grad, float *__restrict__ m,
                            float *__restrict__ v, float lr, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NP) return;
  const float g = grad[q];
  const float mq = 0.9f * m[q] + 0.1f * g;
  const float vq = 0.999f * v[q] + 0.001f * g * g;
  m[q] = mq;
  v[q] = vq;
  P[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
}

static inline size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Work {
  float *P, *m, *v, *grad, *partial, *X, *Y, *out;
  int32_t *idx;
};

static Work carve(void *w, int32_t n, int32_t batch) {
  char *p = static_cast<char *>(w);
  Work k;
  auto take = [&](size_t bytes) {
    char *q = p;
    p += a256(bytes);
    return q;
  };
  const int32_t parts = (std::max(1, std::min(batch, n)) + SB - 1) / SB;
  k.P = reinterpret_cast<float *>(take(sizeof(float) * NP));
  k.m = reinterpret_cast<float *>(take(sizeof(float) * NP));
  k.v = reinterpret_cast<float *>(take(sizeof(float) * NP));
  k.grad = reinterpret_cast<float *>(take(sizeof(float) * NP));
  k.partial = reinterpret_cast<float *>(take(sizeof(float) * NP * (size_t)parts));
  k.X = reinterpret_cast<float *>(take(sizeof(float) * IN * (size_t)n));
  k.Y = reinterpret_cast<float *>(take(sizeof(float) * (size_t)n));
  k.out = reinterpret_cast<float *>(take(sizeof(float) * (size_t)n));
  k.idx = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)n));
  return k;
}

static size_t work_bytes(int32_t n, int32_t batch) {
  const int32_t parts = (std::max(1, std::min(batch, n)) + SB - 1) / SB;
  return 4 * a256(sizeof(float) * NP) + a256(sizeof(float) * NP * (size_t)parts) +
         a256(sizeof(float) * IN * (size_t)n) + 2 * a256(sizeof(float) * (size_t)n) + a256(sizeof(int32_t) * (size_t)n);
}

static void pack(const pjds_mlp &m, float *P) {
  memcpy(P + O_W1, m.w1, sizeof(m.w1));
  memcpy(P + O_B1, m.b1, sizeof(m.b1));
  memcpy(P + O_W2, m.w2, sizeof(m.w2));
  memcpy(P + O_B2, m.b2, sizeof(m.b2));
  memcpy(P + O_W3, m.w3, sizeof(m.w3));
  P[O_B3] = m.b3;
}

static void unpack(const float *P, pjds_mlp &m) {
  memcpy(m.w1, P + O_W1, sizeof(m.w1));
  memcpy(m.b1, P + O_B1, sizeof(m.b1));
  memcpy(m.w2, P + O_W2, sizeof(m.w2));
  memcpy(m.b2, P + O_B2, sizeof(m.b2));
  memcpy(m.w3, P + O_W3, sizeof(m.w3));
  m.b3 = P[O_B3];
}

static inline uint64_t mix64(uint64_t z) {  // splitmix64 output function
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static int set_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(S_GRAD_END * sizeof(float)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_FWD_END * sizeof(float)));
  return e == cudaSuccess ? PJDS_OK : set_error(PJDS_ECUDA, "shared memory attribute: %s", cudaGetErrorString(e));
}

// standardised copy of host inputs
static void standardise(const pjds_mlp &m, const float *X, const float *y, int32_t n, std::vector<float> &Xs,
                        std::vector<float> &ys) {
  Xs.resize((size_t)n * IN);
  for (int64_t s = 0; s < n; ++s)
    for (int i = 0; i < IN; ++i) Xs[(size_t)(s * IN + i)] = (X[s * IN + i] - m.in_mean[i]) / m.in_std[i];
  if (y) {
    ys.resize((size_t)n);
    for (int64_t s = 0; s < n; ++s) ys[(size_t)s] = (y[s] - m.out_mean) / m.out_std;
  }
}

}  // namespace mlp
}  // namespace pjds

using namespace pjds;
using namespace pjds::mlp;

extern "C" int pjds_mlp_init(pjds_mlp *m, uint64_t seed) {
  clear_error();
  if (!m) return set_error(PJDS_EINVAL, "m is NULL");
  memset(m, 0, sizeof(*m));
  uint64_t c = 0;
  auto u = [&](float lim) {
    const uint64_t r = mix64(mix64(seed * 0x9E3779B97F4A7C15ULL + 77) + (c++) * 0xD1B54A32D192ED03ULL);
    return (float)(((double)(r >> 11) * 0x1.0p-53 * 2.0 - 1.0) * lim);
  };
  const float l1 = sqrtf(6.0f / IN), l2 = sqrtf(6.0f / H);
  for (float &w : m->w1) w = u(l1);
  for (float &w : m->w2) w = u(l2);
  for (float &w : m->w3) w = u(l2);
  for (int i = 0; i < IN; ++i) m->in_std[i] = 1.0f;
  m->out_std = 1.0f;
  for (int i = 0; i < PJDS_MLP_FEATURES; ++i) {
    m->feat_lo[i] = 1.0f;
    m->feat_hi[i] = -1.0f;
  }
  return PJDS_OK;
}

extern "C" int pjds_mlp_fit_range(pjds_mlp *m, const float *feat, int32_t n) {
  clear_error();
  if (!m || !feat || n <= 0) return set_error(PJDS_EINVAL, "bad arguments");
  for (int i = 0; i < PJDS_MLP_FEATURES; ++i) {
    float lo = feat[i], hi = feat[i];
    for (int64_t k = 1; k < n; ++k) {
      lo = std::min(lo, feat[k * PJDS_MLP_FEATURES + i]);
      hi = std::max(hi, feat[k * PJDS_MLP_FEATURES + i]);
    }
    m->feat_lo[i] = lo;
    m->feat_hi[i] = hi;
  }
  return PJDS_OK;
}

extern "C" int pjds_mlp_fit_scaling(pjds_mlp *m, const float *X, const float *y, int32_t n) {
  clear_error();
  if (!m || !X || !y || n <= 0) return set_error(PJDS_EINVAL, "bad arguments");
  for (int i = 0; i < IN; ++i) {
    double s = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < n; ++k) s += X[k * IN + i];
    const double mu = s / n;
    for (int64_t k = 0; k < n; ++k) s2 += (X[k * IN + i] - mu) * (X[k * IN + i] - mu);
    const double sd = sqrt(s2 / n);
    m->in_mean[i] = (float)mu;
    m->in_std[i] = sd > 1e-12 ? (float)sd : 1.0f;
  }
  double s = 0.0, s2 = 0.0;
  for (int64_t k = 0; k < n; ++k) s += y[k];
  const double mu = s / n;
  for (int64_t k = 0; k < n; ++k) s2 += (y[k] - mu) * (y[k] - mu);
  const double sd = sqrt(s2 / n);
  m->out_mean = (float)mu;
  m->out_std = sd > 1e-12 ? (float)sd : 1.0f;
  return PJDS_OK;
}

extern "C" int pjds_mlp_workspace_bytes(int32_t n, int32_t batch, size_t *bytes) {
  clear_error();
  if (n <= 0 || batch <= 0 || !bytes) return set_error(PJDS_EINVAL, "bad arguments");
  *bytes = work_bytes(n, batch);
  return PJDS_OK;
}

extern "C" int pjds_mlp_train(pjds_mlp *m, const float *X, const float *y, int32_t n, int32_t epochs, int32_t batch,
                              float lr, uint64_t seed, float *loss_hist, void *work, size_t wbytes, void *stream) {
  clear_error();
  if (!m || !X || !y || !work || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.0f))
    return set_error(PJDS_EINVAL, "bad arguments");
  if (wbytes < work_bytes(n, batch)) return set_error(PJDS_EINVAL, "workspace too small");
  int rc = set_smem_limits();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t bsz = std::min(batch, n);
  Work w = carve(work, n, batch);
  std::vector<float> Xs, ys, P(NP);
  standardise(*m, X, y, n, Xs, ys);
  pack(*m, P.data());
  std::vector<int32_t> order((size_t)n);
  for (int32_t i = 0; i < n; ++i) order[(size_t)i] = i;
  cudaError_t e = cudaMemcpyAsync(w.X, Xs.data(), sizeof(float) * Xs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.Y, ys.data(), sizeof(float) * ys.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.P, P.data(), sizeof(float) * NP, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.m, 0, sizeof(float) * NP, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.v, 0, sizeof(float) * NP, s);
  if (e == cudaSuccess && bsz >= n)
    e = cudaMemcpyAsync(w.idx, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp upload: %s", cudaGetErrorString(e));
  std::vector<float> out((size_t)n);
  int64_t t = 0;
  for (int32_t ep = 0; ep < epochs; ++ep) {
    if (bsz < n) {  // Fisher-Yates with a counter-based generator
      for (int32_t i = 0; i < n; ++i) order[(size_t)i] = i;
      for (int32_t i = n - 1; i > 0; --i) {
        const uint64_t r = mix64(mix64(seed + 0x51ED2701ULL * (uint64_t)(ep + 1)) + (uint64_t)i);
        const int32_t j = (int32_t)(r % (uint64_t)(i + 1));
        std::swap(order[(size_t)i], order[(size_t)j]);
      }
      e = cudaMemcpyAsync(w.idx, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host order buffer is reused next epoch
      if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp order upload: %s", cudaGetErrorString(e));
    }
    for (int32_t b0 = 0; b0 < n; b0 += bsz) {
      const int32_t cnt = std::min(bsz, n - b0);
      const int32_t parts = (cnt + SB - 1) / SB;
      grad_kernel<<<parts, NT, S_GRAD_END * sizeof(float), s>>>(w.P, w.X, w.Y, w.idx + b0, cnt, 1.0f / (float)cnt,
                                                                 w.partial);
      reduce_kernel<<<(NP + 255) / 256, 256, 0, s>>>(w.partial, parts, w.grad);
      ++t;
      const float c1 = (float)(1.0 - pow(0.9, (double)t)), c2 = (float)(1.0 - pow(0.999, (double)t));
      adam_kernel<<<(NP + 255) / 256, 256, 0, s>>>(w.P, w.grad, w.m, w.v, lr, c1, c2);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp training launch: %s", cudaGetErrorString(e));
    if (loss_hist) {
      forward_kernel<<<(n + SB - 1) / SB, NT, S_FWD_END * sizeof(float), s>>>(w.P, w.X, n, w.out);
      e = cudaMemcpyAsync(out.data(), w.out, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp loss: %s", cudaGetErrorString(e));
      double acc = 0.0;
      for (int32_t i = 0; i < n; ++i) acc += ((double)out[(size_t)i] - ys[(size_t)i]) * ((double)out[(size_t)i] - ys[(size_t)i]);
      loss_hist[ep] = (float)(acc / n);
    }
  }
  e = cudaMemcpyAsync(P.data(), w.P, sizeof(float) * NP, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp download: %s", cudaGetErrorString(e));
  unpack(P.data(), *m);
  return PJDS_OK;
}

extern "C" int pjds_mlp_predict(const pjds_mlp *m, const float *X, int32_t n, float *out, void *work, size_t wbytes,
                                void *stream) {
  clear_error();
  if (!m || !X || !out || !work || n <= 0) return set_error(PJDS_EINVAL, "bad arguments");
  if (wbytes < work_bytes(n, 1)) return set_error(PJDS_EINVAL, "workspace too small");
  int rc = set_smem_limits();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w = carve(work, n, 1);
  std::vector<float> Xs, ys, P(NP);
  standardise(*m, X, nullptr, n, Xs, ys);
  pack(*m, P.data());
  cudaError_t e = cudaMemcpyAsync(w.X, Xs.data(), sizeof(float) * Xs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.P, P.data(), sizeof(float) * NP, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp upload: %s", cudaGetErrorString(e));
  forward_kernel<<<(n + SB - 1) / SB, NT, S_FWD_END * sizeof(float), s>>>(w.P, w.X, n, w.out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, w.out, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PJDS_ECUDA, "mlp predict: %s", cudaGetErrorString(e));
  for (int32_t i = 0; i < n; ++i) out[i] = out[i] * m->out_std + m->out_mean;
  return PJDS_OK;
}

extern "C" int pjds_features(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                             float out[PJDS_MLP_FEATURES]) {
  clear_error();
  if (n_rows <= 0 || n_cols < 1 || !row_ptr || !out) return set_error(PJDS_EINVAL, "bad arguments");
  const int64_t nnz = row_ptr[n_rows];
  if (nnz > 0 && !col_idx) return set_error(PJDS_EINVAL, "col_idx is NULL");
  double s1 = 0.0, s2 = 0.0, s3 = 0.0, mx = 0.0;
  const double mean = (double)nnz / n_rows;
  for (int32_t i = 0; i < n_rows; ++i) {
    const double l = (double)(row_ptr[i + 1] - row_ptr[i]), d = l - mean;
    s1 += l;
    s2 += d * d;
    s3 += d * d * d;
    mx = std::max(mx, l);
  }
  const double var = s2 / n_rows, sd = sqrt(var);
  double band = 0.0, near = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : band, near)
  for (int32_t i = 0; i < n_rows; ++i)
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double d = fabs((double)col_idx[k] - (double)i);
      band += d;
      near += d <= 64.0 ? 1.0 : 0.0;
    }
  out[0] = (float)log10((double)n_rows);
  out[1] = (float)log10((double)std::max<int64_t>(nnz, 1));
  out[2] = (float)log2(1.0 + mean);
  out[3] = mean > 0.0 ? (float)(sd / mean) : 0.0f;
  out[4] = sd > 0.0 ? (float)((s3 / n_rows) / (sd * sd * sd)) : 0.0f;
  out[5] = (float)log2(1.0 + mx);
  out[6] = nnz > 0 ? (float)(band / nnz / n_rows) : 0.0f;
  out[7] = nnz > 0 ? (float)(near / nnz) : 0.0f;
  (void)s1;
  return PJDS_OK;
}

extern "C" int pjds_tune_encode(const float feat[PJDS_MLP_FEATURES], const pjds_candidate *cands, int32_t n,
                                float *out) {
  clear_error();
  if (!feat || !cands || !out || n <= 0) return set_error(PJDS_EINVAL, "bad arguments");
  for (int32_t c = 0; c < n; ++c) {
    float *o = out + (int64_t)c * IN;
    for (int i = 0; i < PJDS_MLP_FEATURES; ++i) o[i] = feat[i];
    const bool plan = cands[c].plan == 1;
    const int32_t t = !plan && cands[c].threads_per_row > 0 ? cands[c].threads_per_row : 1;
    o[8] = (float)log2((double)cands[c].b / 32.0);
    o[9] = (float)log2((double)t);
    o[10] = cands[c].dtype == PJDS_F64 ? 1.0f : 0.0f;
    o[11] = cands[c].dtype == PJDS_F32 ? 1.0f : 0.0f;
    o[12] = cands[c].dtype == PJDS_BF16 ? 1.0f : 0.0f;
    o[13] = plan ? 1.0f : 0.0f;
    o[14] = !plan && cands[c].tile_order == 1 ? 1.0f : 0.0f;
  }
  return PJDS_OK;
}

extern "C" int pjds_tune_pick(int32_t n_rows, int32_t n_cols, const int64_t *row_ptr, const int32_t *col_idx,
                              const double *val, const pjds_mlp *model, const pjds_candidate *cands, int32_t n_cands,
                              int32_t reps, void *work, size_t work_bytes, void *arena, size_t arena_bytes,
                              void *flush, size_t flush_bytes, pjds_pick *out, void *stream) {
  clear_error();
  if (!out || !cands || n_cands <= 0 || !row_ptr || n_rows <= 0 || n_cols < 1)
    return set_error(PJDS_EINVAL, "bad arguments");
  memset(out, 0, sizeof(*out));
  float feat[PJDS_MLP_FEATURES];
  int rc = pjds_features(n_rows, n_cols, row_ptr, col_idx, feat);
  if (rc) return rc;
  int32_t outside = 0;
  if (model) {
    for (int i = 0; i < PJDS_MLP_FEATURES; ++i) {
      const float lo = model->feat_lo[i], hi = model->feat_hi[i];
      if (lo > hi) continue;  // no range: trusted
      const float tol = 0.02f * (hi - lo);
      outside += feat[i] < lo - tol || feat[i] > hi + tol;
    }
  }
  out->n_outside = outside;
  if (model && outside == 0) {
    std::vector<float> X((size_t)n_cands * IN), pred((size_t)n_cands);
    if ((rc = pjds_tune_encode(feat, cands, n_cands, X.data()))) return rc;
    if ((rc = pjds_mlp_predict(model, X.data(), n_cands, pred.data(), work, work_bytes, stream))) return rc;
    int32_t best = 0;
    for (int32_t c = 1; c < n_cands; ++c)
      if (pred[(size_t)c] < pred[(size_t)best]) best = c;
    out->cand = cands[best];
    out->index = best;
    out->source = PJDS_PICK_MODEL;
    out->us = exp((double)pred[(size_t)best]);
    return PJDS_OK;
  }
  if (!arena) return set_error(PJDS_EINVAL, "the matrix lies outside the model's range and no sweep arena was given");
  std::vector<pjds_tune_entry> e((size_t)n_cands);
  int32_t best = -1;
  rc = pjds_tune_sweep(n_rows, n_cols, row_ptr, col_idx, val, cands, n_cands, reps, arena, arena_bytes, flush,
                       flush_bytes, e.data(), &best, stream);
  if (rc) return rc;
  if (best < 0) return set_error(PJDS_EINVAL, "no candidate ran");
  out->cand = cands[best];
  out->index = best;
  out->source = PJDS_PICK_SWEEP;
  out->us = e[(size_t)best].us;
  clear_error();
  return PJDS_OK;
}
