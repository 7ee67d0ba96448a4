// The cover/plan chooser's network: a three-layer perceptron
// y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 trained by plain gradient
// descent on the mean squared error, with its own forward, backward and
// update kernels (no library GEMM: the layers are at most 128 wide and the
// batches a few thousand rows, so one thread per output element is enough
// and the whole step stays on the context's stream).
//
// Parameter layout (float32, one contiguous device array): W1 (h1 x d,
// row-major), b1 (h1), W2 (h2 x h1), b2 (h2), W3 (1 x h2), b3 (1).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fj.h"
#include <algorithm>

#include "fj_ctx_access.h"

namespace {

constexpr int kT = 256;

struct Layout {
  int d, h1, h2;
  size_t w1, b1, w2, b2, w3, b3, n;
  Layout(int d_, int h1_, int h2_) : d(d_), h1(h1_), h2(h2_) {
    w1 = 0;
    b1 = w1 + size_t(h1) * d;
    w2 = b1 + h1;
    b2 = w2 + size_t(h2) * h1;
    w3 = b2 + h2;
    b3 = w3 + h2;
    n = b3 + 1;
  }
};

// Z = X W^T + b (n x out), A = relu(Z) when `relu` (else A = Z).
__global__ void k_dense_fwd(const float* __restrict__ x, int n, int in,
                            const float* __restrict__ w, const float* __restrict__ b, int out,
                            float* __restrict__ z, float* __restrict__ a, int relu) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * out) return;
  const int r = idx / out, o = idx % out;
  const float* xr = x + size_t(r) * in;
  const float* wo = w + size_t(o) * in;
  float s = b[o];
  for (int i = 0; i < in; ++i) s = fmaf(xr[i], wo[i], s);
  z[idx] = s;
  a[idx] = relu ? fmaxf(s, 0.f) : s;
}

// dy = 2 (y - t) / n, and the summed squared error into *sse.
__global__ void k_mse_grad(const float* __restrict__ y, const float* __restrict__ t, int n,
                           float* __restrict__ dy, float* __restrict__ sse) {
  __shared__ float sh[kT];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (i < n) {
    e = y[i] - t[i];
    dy[i] = 2.f * e / float(n);
  }
  sh[threadIdx.x] = e * e;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(sse, sh[0]);
}

// dW[o][i] = sum_r dZ[r][o] A[r][i] and db[o] = sum_r dZ[r][o]: one thread
// per weight (i == in: the bias).
__global__ void k_dense_bwd_w(const float* __restrict__ dz, const float* __restrict__ a, int n,
                              int in, int out, float* __restrict__ dw, float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= out * (in + 1)) return;
  const int o = idx / (in + 1), i = idx % (in + 1);
  float s = 0.f;
  if (i < in) {
    for (int r = 0; r < n; ++r) s = fmaf(dz[size_t(r) * out + o], a[size_t(r) * in + i], s);
    dw[size_t(o) * in + i] = s;
  } else {
    for (int r = 0; r < n; ++r) s += dz[size_t(r) * out + o];
    db[o] = s;
  }
}

// dZprev[r][i] = (sum_o dZ[r][o] W[o][i]) * [Zprev[r][i] > 0].
__global__ void k_dense_bwd_x(const float* __restrict__ dz, const float* __restrict__ w, int n,
                              int in, int out, const float* __restrict__ zprev,
                              float* __restrict__ dzprev) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * in) return;
  const int r = idx / in, i = idx % in;
  float s = 0.f;
  for (int o = 0; o < out; ++o) s = fmaf(dz[size_t(r) * out + o], w[size_t(o) * in + i], s);
  dzprev[idx] = zprev[idx] > 0.f ? s : 0.f;
}

__global__ void k_sgd(float* __restrict__ p, const float* __restrict__ g, size_t n, float lr) {
  const size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (i < n) p[i] -= lr * g[i];
}

int blocks(size_t n) { return int((n + kT - 1) / kT); }

thread_local std::string g_model_err;

}  // namespace

struct fj_model {
  fj_ctx* ctx = nullptr;
  Layout L{1, 1, 1};
  int max_batch = 0;
  float* params = nullptr;
  float* grads = nullptr;
  float* z1 = nullptr;  // n x h1 (and relu copies)
  float* a1 = nullptr;
  float* z2 = nullptr;  // n x h2
  float* a2 = nullptr;
  float* y = nullptr;   // n
  float* dy = nullptr;  // n
  float* dz2 = nullptr;
  float* dz1 = nullptr;
  float* sse = nullptr;
  float* h_sse = nullptr;  // pinned
  // Feature scaler used by the chooser: x' = (x - mean) / scale per input
  // (empty: identity).
  std::vector<float> mean, scale;
};

namespace {

fj_status model_fail(fj_status st, const std::string& m) {
  g_model_err = m;
  return st;
}

fj_status ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FJ_OK;
  return model_fail(FJ_ERR_CUDA, std::string("CUDA: ") + what + ": " + cudaGetErrorString(e));
}

#define MCK(x)                                   \
  do {                                           \
    fj_status st_ = ck((x), #x);                 \
    if (st_ != FJ_OK) return st_;                \
  } while (0)

fj_status forward(fj_model* m, const float* x, int n) {
  const Layout& L = m->L;
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  const float* p = m->params;
  k_dense_fwd<<<blocks(size_t(n) * L.h1), kT, 0, s>>>(x, n, L.d, p + L.w1, p + L.b1, L.h1, m->z1,
                                                      m->a1, 1);
  k_dense_fwd<<<blocks(size_t(n) * L.h2), kT, 0, s>>>(m->a1, n, L.h1, p + L.w2, p + L.b2, L.h2,
                                                      m->z2, m->a2, 1);
  k_dense_fwd<<<blocks(size_t(n)), kT, 0, s>>>(m->a2, n, L.h2, p + L.w3, p + L.b3, 1, m->y, m->y,
                                               0);
  return ck(cudaGetLastError(), "model forward");
}

// Gradients of the mean squared error into m->grads; the summed squared
// error into m->sse (device).
fj_status backward(fj_model* m, const float* x, const float* t, int n) {
  const Layout& L = m->L;
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  float* g = m->grads;
  const float* p = m->params;
  MCK(cudaMemsetAsync(m->sse, 0, sizeof(float), s));
  k_mse_grad<<<blocks(size_t(n)), kT, 0, s>>>(m->y, t, n, m->dy, m->sse);
  k_dense_bwd_w<<<blocks(size_t(L.h2) + 1), kT, 0, s>>>(m->dy, m->a2, n, L.h2, 1, g + L.w3,
                                                        g + L.b3);
  k_dense_bwd_x<<<blocks(size_t(n) * L.h2), kT, 0, s>>>(m->dy, p + L.w3, n, L.h2, 1, m->z2, m->dz2);
  k_dense_bwd_w<<<blocks(size_t(L.h2) * (L.h1 + 1)), kT, 0, s>>>(m->dz2, m->a1, n, L.h1, L.h2,
                                                                 g + L.w2, g + L.b2);
  k_dense_bwd_x<<<blocks(size_t(n) * L.h1), kT, 0, s>>>(m->dz2, p + L.w2, n, L.h1, L.h2, m->z1,
                                                        m->dz1);
  k_dense_bwd_w<<<blocks(size_t(L.h1) * (L.d + 1)), kT, 0, s>>>(m->dz1, x, n, L.d, L.h1, g + L.w1,
                                                                g + L.b1);
  return ck(cudaGetLastError(), "model backward");
}

fj_status check_batch(const fj_model* m, const void* x, int n) {
  if (!m) return model_fail(FJ_ERR_INVALID_ARG, "NULL model");
  if (n < 0 || n > m->max_batch)
    return model_fail(FJ_ERR_INVALID_ARG, "batch of " + std::to_string(n) + " rows above the model's " +
                                              std::to_string(m->max_batch));
  if (n > 0 && !x) return model_fail(FJ_ERR_INVALID_ARG, "NULL input");
  return FJ_OK;
}

}  // namespace

extern "C" {

const char* fj_model_last_error(void) { return g_model_err.c_str(); }

fj_status fj_model_create(fj_ctx* ctx, int in_dim, int h1, int h2, int max_batch,
                          fj_model** out) {
  g_model_err.clear();
  if (!ctx || !out || in_dim < 1 || h1 < 1 || h2 < 1 || max_batch < 1 || in_dim > 4096 ||
      h1 > 4096 || h2 > 4096)
    return model_fail(FJ_ERR_INVALID_ARG, "bad model shape");
  fj_model* m = new fj_model;
  m->ctx = ctx;
  m->L = Layout(in_dim, h1, h2);
  m->max_batch = max_batch;
  MCK(cudaSetDevice(fj_internal_ctx_device(ctx)));
  const size_t nb = size_t(max_batch);
  float** bufs[] = {&m->params, &m->grads, &m->z1, &m->a1, &m->z2, &m->a2,
                    &m->y,      &m->dy,    &m->dz2, &m->dz1, &m->sse};
  const size_t sizes[] = {m->L.n, m->L.n, nb * h1, nb * h1, nb * h2, nb * h2,
                          nb,     nb,     nb * h2, nb * h1, 1};
  for (int i = 0; i < 11; ++i) {
    cudaError_t e = cudaMalloc(bufs[i], sizes[i] * sizeof(float));
    if (e != cudaSuccess) {
      fj_model_free(m);
      return model_fail(FJ_ERR_OOM, "model buffers");
    }
  }
  if (cudaMallocHost(&m->h_sse, sizeof(float)) != cudaSuccess) {
    fj_model_free(m);
    return model_fail(FJ_ERR_OOM, "model host buffer");
  }
  cudaStream_t s = fj_internal_ctx_stream(ctx);
  MCK(cudaMemsetAsync(m->params, 0, m->L.n * sizeof(float), s));
  *out = m;
  return FJ_OK;
}

size_t fj_model_n_params(const fj_model* m) { return m ? m->L.n : 0; }

fj_status fj_model_set_params(fj_model* m, const float* host, size_t n) {
  if (!m || !host || n != m->L.n) return model_fail(FJ_ERR_INVALID_ARG, "parameter count");
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  MCK(cudaMemcpyAsync(m->params, host, n * sizeof(float), cudaMemcpyHostToDevice, s));
  MCK(cudaStreamSynchronize(s));
  return FJ_OK;
}

fj_status fj_model_get_params(fj_model* m, float* host, size_t n) {
  if (!m || !host || n != m->L.n) return model_fail(FJ_ERR_INVALID_ARG, "parameter count");
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  MCK(cudaMemcpyAsync(host, m->params, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return FJ_OK;
}

fj_status fj_model_forward(fj_model* m, const float* d_x, int n, float* d_y) {
  fj_status st = check_batch(m, d_x, n);
  if (st != FJ_OK) return st;
  if (n == 0) return FJ_OK;
  if (!d_y) return model_fail(FJ_ERR_INVALID_ARG, "NULL output");
  st = forward(m, d_x, n);
  if (st != FJ_OK) return st;
  return ck(cudaMemcpyAsync(d_y, m->y, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice,
                            fj_internal_ctx_stream(m->ctx)),
            "model output copy");
}

fj_status fj_model_gradients(fj_model* m, const float* d_x, const float* d_t, int n,
                             float* host_grads, float* host_loss) {
  fj_status st = check_batch(m, d_x, n);
  if (st != FJ_OK) return st;
  if (n == 0 || !d_t || !host_grads) return model_fail(FJ_ERR_INVALID_ARG, "empty batch or NULL");
  if ((st = forward(m, d_x, n)) != FJ_OK || (st = backward(m, d_x, d_t, n)) != FJ_OK) return st;
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  MCK(cudaMemcpyAsync(host_grads, m->grads, m->L.n * sizeof(float), cudaMemcpyDeviceToHost, s));
  MCK(cudaMemcpyAsync(m->h_sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  if (host_loss) *host_loss = *m->h_sse / float(n);
  return FJ_OK;
}

fj_status fj_model_train_step(fj_model* m, const float* d_x, const float* d_t, int n, float lr,
                              float* host_loss) {
  fj_status st = check_batch(m, d_x, n);
  if (st != FJ_OK) return st;
  if (n == 0 || !d_t) return model_fail(FJ_ERR_INVALID_ARG, "empty batch or NULL target");
  if ((st = forward(m, d_x, n)) != FJ_OK || (st = backward(m, d_x, d_t, n)) != FJ_OK) return st;
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  k_sgd<<<blocks(m->L.n), kT, 0, s>>>(m->params, m->grads, m->L.n, lr);
  MCK(cudaGetLastError());
  if (host_loss) {
    MCK(cudaMemcpyAsync(m->h_sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    *host_loss = *m->h_sse / float(n);
  }
  return FJ_OK;
}

fj_status fj_model_set_scaler(fj_model* m, const float* mean, const float* scale, size_t n) {
  if (!m || n != size_t(m->L.d) || !mean || !scale)
    return model_fail(FJ_ERR_INVALID_ARG, "scaler needs in_dim means and scales");
  for (size_t i = 0; i < n; ++i)
    if (!(scale[i] > 0.f)) return model_fail(FJ_ERR_INVALID_ARG, "scales must be positive");
  m->mean.assign(mean, mean + n);
  m->scale.assign(scale, scale + n);
  return FJ_OK;
}

// File layout (little-endian, as written by this library): 8 bytes
// "FJMLP001"; int32 in_dim, h1, h2, has_scaler; the parameters (float32, the
// model's layout); then, when has_scaler, in_dim means and in_dim scales.
fj_status fj_model_save(fj_model* m, const char* path) {
  if (!m || !path) return model_fail(FJ_ERR_INVALID_ARG, "NULL model or path");
  std::vector<float> p(m->L.n);
  fj_status st = fj_model_get_params(m, p.data(), p.size());
  if (st != FJ_OK) return st;
  FILE* f = fopen(path, "wb");
  if (!f) return model_fail(FJ_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const int32_t hdr[4] = {m->L.d, m->L.h1, m->L.h2, m->mean.empty() ? 0 : 1};
  bool ok = fwrite("FJMLP001", 1, 8, f) == 8 && fwrite(hdr, 4, 4, f) == 4 &&
            fwrite(p.data(), 4, p.size(), f) == p.size();
  if (ok && hdr[3])
    ok = fwrite(m->mean.data(), 4, m->mean.size(), f) == m->mean.size() &&
         fwrite(m->scale.data(), 4, m->scale.size(), f) == m->scale.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? FJ_OK : model_fail(FJ_ERR_INVALID_ARG, std::string("short write to ") + path);
}

fj_status fj_model_load(fj_ctx* ctx, const char* path, int max_batch, fj_model** out) {
  if (!ctx || !path || !out) return model_fail(FJ_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return model_fail(FJ_ERR_INVALID_ARG, std::string("cannot read ") + path);
  char magic[8];
  int32_t hdr[4];
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "FJMLP001", 8) != 0 ||
      fread(hdr, 4, 4, f) != 4 || hdr[0] < 1 || hdr[1] < 1 || hdr[2] < 1 || hdr[0] > 4096 ||
      hdr[1] > 4096 || hdr[2] > 4096 || (hdr[3] != 0 && hdr[3] != 1)) {
    fclose(f);
    return model_fail(FJ_ERR_INVALID_ARG, std::string("not a model file: ") + path);
  }
  Layout L(hdr[0], hdr[1], hdr[2]);
  std::vector<float> p(L.n), mean, scale;
  bool ok = fread(p.data(), 4, p.size(), f) == p.size();
  if (ok && hdr[3]) {
    mean.resize(hdr[0]);
    scale.resize(hdr[0]);
    ok = fread(mean.data(), 4, mean.size(), f) == mean.size() &&
         fread(scale.data(), 4, scale.size(), f) == scale.size();
  }
  fclose(f);
  if (!ok) return model_fail(FJ_ERR_INVALID_ARG, std::string("truncated model file: ") + path);
  fj_model* m = nullptr;
  fj_status st = fj_model_create(ctx, hdr[0], hdr[1], hdr[2], max_batch, &m);
  if (st != FJ_OK) return st;
  if ((st = fj_model_set_params(m, p.data(), p.size())) != FJ_OK ||
      (hdr[3] && (st = fj_model_set_scaler(m, mean.data(), scale.data(), mean.size())) != FJ_OK)) {
    fj_model_free(m);
    return st;
  }
  *out = m;
  return FJ_OK;
}

void fj_model_free(fj_model* m) {
  if (!m) return;
  if (m->ctx) cudaStreamSynchronize(fj_internal_ctx_stream(m->ctx));
  float* bufs[] = {m->params, m->grads, m->z1, m->a1, m->z2, m->a2,
                   m->y,      m->dy,    m->dz2, m->dz1, m->sse};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (m->h_sse) cudaFreeHost(m->h_sse);
  delete m;
}

}  // extern "C"

fj_status fj_internal_model_predict(fj_model* m, const float* host_x, int n, int dim,
                                    float* host_y) {
  if (!m || dim != m->L.d) return model_fail(FJ_ERR_INVALID_ARG, "feature width differs from the model's");
  std::vector<float> x(host_x, host_x + size_t(n) * dim);
  if (!m->mean.empty())
    for (int r = 0; r < n; ++r)
      for (int i = 0; i < dim; ++i)
        x[size_t(r) * dim + i] = (x[size_t(r) * dim + i] - m->mean[i]) / m->scale[i];
  cudaStream_t s = fj_internal_ctx_stream(m->ctx);
  for (int r0 = 0; r0 < n; r0 += m->max_batch) {
    const int k = std::min(m->max_batch, n - r0);
    // The standardized rows go to a device buffer of their own (host-side
    // planning code, outside any captured or timed region).
    float* d_x = nullptr;
    MCK(cudaMalloc(&d_x, size_t(k) * dim * sizeof(float)));
    fj_status st = ck(cudaMemcpyAsync(d_x, x.data() + size_t(r0) * dim, size_t(k) * dim * sizeof(float),
                                      cudaMemcpyHostToDevice, s), "features to the device");
    if (st == FJ_OK) st = forward(m, d_x, k);
    if (st == FJ_OK)
      st = ck(cudaMemcpyAsync(host_y + r0, m->y, size_t(k) * sizeof(float),
                              cudaMemcpyDeviceToHost, s), "predictions to the host");
    if (st == FJ_OK) st = ck(cudaStreamSynchronize(s), "prediction");
    cudaFree(d_x);
    if (st != FJ_OK) return st;
  }
  return FJ_OK;
}
