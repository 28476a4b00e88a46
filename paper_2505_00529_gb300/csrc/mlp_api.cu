// C ABI of the learned warm start (see mlp.cu for the kernels): parameters,
// Adam state, a device-resident training set, minibatch training, the loss
// gradient (for checks against an independent implementation) and
// inference with bfloat16 weights.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.hpp"
#include "qoc.h"

namespace qoc {
cudaError_t mlp_gemm(const float* A, long sam, long sak, const void* B, int b_bf16, long sbk,
                     long sbn, float* C, long scm, int M, int N, int K, int mode, const float* bias,
                     float* pre, const float* pre_in, int accumulate, cudaStream_t st);
cudaError_t mlp_colsum(const float* dY, int Bn, int N, float* db, cudaStream_t st);
cudaError_t mlp_mse(const float* Y, const float* T, int n, float inv_b, float* dY, float* loss,
                    cudaStream_t st);
cudaError_t mlp_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                     float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t mlp_to_bf16(const float* x, void* y, int n, cudaStream_t st);
cudaError_t mlp_gemm_bf16_tc(const float* A, long sam, long sak, const void* B, long sbk, long sbn,
                             float* C, long scm, int M, int N, int K, int mode, const float* bias,
                             cudaStream_t st);
cudaError_t mlp_gather(const float* src, const int* idx, int rows, int cols, float* dst,
                       cudaStream_t st);
}  // namespace qoc

using namespace qoc;

struct qoc_mlp {
  int L = 0;                      // linear layers (hidden layers + 1)
  std::vector<int> d;             // widths d[0..L]
  std::vector<size_t> woff, boff; // parameter offsets
  size_t np = 0;
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  void* wbf = nullptr;            // bfloat16 copy for inference
  int bf_valid = 0;
  std::vector<float*> h, pre, dh; // activations [L+1], pre-activations [L], gradients [L+1]
  float* loss = nullptr;
  float *X = nullptr, *T = nullptr; // dataset
  int n_data = 0;
  int* perm = nullptr;
  int adam_t = 0;
  float* hbuf = nullptr;          // pinned staging
  size_t hbuf_len = 0;
};

namespace {
qoc_status cu(cudaError_t e) {
  if (e == cudaSuccess) return QOC_OK;
  return e == cudaErrorMemoryAllocation ? QOC_ENOMEM : QOC_ECUDA;
}
#define MTRY(x)                              \
  do {                                       \
    qoc_status s_ = cu(x);                   \
    if (s_ != QOC_OK) return s_;             \
  } while (0)

size_t count_params(int n_in, int hidden, int nh, int n_out) {
  size_t n = 0;
  int a = n_in;
  for (int k = 0; k < nh; ++k) { n += (size_t)a * hidden + hidden; a = hidden; }
  return n + (size_t)a * n_out + n_out;
}

// forward pass on rows X (batch x d0) into p->h; inference=1 uses the bf16 weights
qoc_status forward(qoc_mlp* p, const float* X, int B, int bf16) {
  const float* in = X;
  for (int k = 0; k < p->L; ++k) {
    const int a = p->d[k], b = p->d[k + 1];
    const bool last = k == p->L - 1;
    if (bf16) {   // inference on the tensor cores: bfloat16 weights and activations
      const void* W = (const void*)((const unsigned short*)p->wbf + p->woff[k]);
      MTRY(mlp_gemm_bf16_tc(in, a, 1, W, b, 1, p->h[k + 1], b, B, b, a, last ? 2 : 1, p->w + p->boff[k],
                            p->stream));
    } else {
      MTRY(mlp_gemm(in, a, 1, p->w + p->woff[k], 0, b, 1, p->h[k + 1], b, B, b, a, last ? 2 : 1,
                    p->w + p->boff[k], p->pre[k], nullptr, 0, p->stream));
    }
    in = p->h[k + 1];
  }
  return QOC_OK;
}

// loss and full gradient into p->g for rows (X, T)
qoc_status backward(qoc_mlp* p, const float* X, const float* T, int B) {
  const int L = p->L;
  MTRY(cudaMemsetAsync(p->loss, 0, sizeof(float), p->stream));
  MTRY(mlp_mse(p->h[L], T, B * p->d[L], 1.0f / B, p->dh[L], p->loss, p->stream));
  for (int k = L - 1; k >= 0; --k) {
    const int a = p->d[k], b = p->d[k + 1];
    const float* hin = k == 0 ? X : p->h[k];
    // dW_k = h_k^T dPre_k   (a x b), db_k = colsum(dPre_k)
    MTRY(mlp_gemm(hin, 1, a, p->dh[k + 1], 0, b, 1, p->g + p->woff[k], b, a, b, B, 0, nullptr,
                  nullptr, nullptr, 0, p->stream));
    MTRY(mlp_colsum(p->dh[k + 1], B, b, p->g + p->boff[k], p->stream));
    if (k > 0) {
      // dPre_{k-1} = (dPre_k W_k^T) o gelu'(pre_{k-1})
      MTRY(mlp_gemm(p->dh[k + 1], b, 1, p->w + p->woff[k], 0, 1, b, p->dh[k], a, B, a, b, 3, nullptr,
                    nullptr, p->pre[k - 1], 0, p->stream));
    }
  }
  return QOC_OK;
}
}  // namespace

extern "C" {

size_t qoc_mlp_param_count(int n_in, int hidden, int n_hidden_layers, int n_out) {
  if (n_in < 1 || hidden < 1 || n_hidden_layers < 0 || n_out < 1) return 0;
  return count_params(n_in, hidden, n_hidden_layers, n_out);
}

void qoc_mlp_destroy(qoc_mlp* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  cudaFree(p->w); cudaFree(p->g); cudaFree(p->m); cudaFree(p->v); cudaFree(p->wbf);
  for (float* x : p->h) cudaFree(x);
  for (float* x : p->pre) cudaFree(x);
  for (float* x : p->dh) cudaFree(x);
  cudaFree(p->loss); cudaFree(p->X); cudaFree(p->T); cudaFree(p->perm);
  if (p->hbuf) cudaFreeHost(p->hbuf);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

qoc_status qoc_mlp_create(int n_in, int hidden, int n_hidden_layers, int n_out,
                          const float* params_init, int max_batch, void* cuda_stream,
                          qoc_mlp** out) {
  if (!out || !params_init) return QOC_EINVAL;
  *out = nullptr;
  if (n_in < 1 || hidden < 1 || n_hidden_layers < 0 || n_out < 1 || max_batch < 1 ||
      n_in > 65536 || hidden > 65536 || n_out > 65536 || n_hidden_layers > 16)
    return QOC_EINVAL;
  qoc_mlp* p = new (std::nothrow) qoc_mlp();
  if (!p) return QOC_ENOMEM;
  p->L = n_hidden_layers + 1;
  p->d.push_back(n_in);
  for (int k = 0; k < n_hidden_layers; ++k) p->d.push_back(hidden);
  p->d.push_back(n_out);
  size_t off = 0;
  for (int k = 0; k < p->L; ++k) {
    p->woff.push_back(off);
    off += (size_t)p->d[k] * p->d[k + 1];
    p->boff.push_back(off);
    off += p->d[k + 1];
  }
  p->np = off;
  for (size_t i = 0; i < p->np; ++i)
    if (!std::isfinite(params_init[i])) { delete p; return QOC_EINVAL; }
  p->max_batch = max_batch;
  auto fail = [&](cudaError_t e) { qoc_mlp_destroy(p); return cu(e); };
  cudaError_t e;
  if (cuda_stream) p->stream = (cudaStream_t)cuda_stream;
  else {
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    p->own_stream = true;
  }
  const size_t nb = p->np * sizeof(float);
  if ((e = cudaMalloc(&p->w, nb)) || (e = cudaMalloc(&p->g, nb)) || (e = cudaMalloc(&p->m, nb)) ||
      (e = cudaMalloc(&p->v, nb)) || (e = cudaMalloc(&p->wbf, p->np * 2)) ||
      (e = cudaMalloc(&p->loss, sizeof(float))))
    return fail(e);
  p->h.assign(p->L + 1, nullptr);
  p->dh.assign(p->L + 1, nullptr);
  p->pre.assign(p->L, nullptr);
  for (int k = 0; k <= p->L; ++k) {
    if ((e = cudaMalloc(&p->h[k], sizeof(float) * (size_t)max_batch * p->d[k])) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dh[k], sizeof(float) * (size_t)max_batch * p->d[k])) != cudaSuccess) return fail(e);
    if (k < p->L && (e = cudaMalloc(&p->pre[k], sizeof(float) * (size_t)max_batch * p->d[k + 1])) != cudaSuccess)
      return fail(e);
  }
  p->hbuf_len = p->np + 64;
  if ((e = cudaMallocHost(&p->hbuf, sizeof(float) * p->hbuf_len)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->w, params_init, nb, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(p->m, 0, nb)) != cudaSuccess || (e = cudaMemset(p->v, 0, nb)) != cudaSuccess)
    return fail(e);
  *out = p;
  return QOC_OK;
}

qoc_status qoc_mlp_get_params(const qoc_mlp* p, float* params) {
  if (!p || !params) return QOC_EINVAL;
  MTRY(cudaStreamSynchronize(p->stream));
  return cu(cudaMemcpy(params, p->w, p->np * sizeof(float), cudaMemcpyDeviceToHost));
}

qoc_status qoc_mlp_set_dataset(qoc_mlp* p, const float* X, const float* T, int n) {
  if (!p || !X || !T || n < 1) return QOC_EINVAL;
  MTRY(cudaStreamSynchronize(p->stream));
  cudaFree(p->X); cudaFree(p->T); cudaFree(p->perm);
  p->X = p->T = nullptr; p->perm = nullptr; p->n_data = 0;
  MTRY(cudaMalloc(&p->X, sizeof(float) * (size_t)n * p->d[0]));
  MTRY(cudaMalloc(&p->T, sizeof(float) * (size_t)n * p->d[p->L]));
  MTRY(cudaMalloc(&p->perm, sizeof(int) * (size_t)n));
  MTRY(cudaMemcpy(p->X, X, sizeof(float) * (size_t)n * p->d[0], cudaMemcpyHostToDevice));
  MTRY(cudaMemcpy(p->T, T, sizeof(float) * (size_t)n * p->d[p->L], cudaMemcpyHostToDevice));
  p->n_data = n;
  return QOC_OK;
}

// One epoch per entry of `perm` (epochs x n sample indices, host): minibatches
// of `batch` rows in that order; Adam with (lr, 0.9, 0.999, 1e-8).  losses
// receives the mean minibatch loss of each epoch.
qoc_status qoc_mlp_train(qoc_mlp* p, const int* perm, int epochs, int batch, float lr, float* losses) {
  if (!p || !perm || !losses || epochs < 1 || batch < 1 || batch > p->max_batch || p->n_data < 1 ||
      !(lr > 0))
    return QOC_EINVAL;
  const int n = p->n_data;
  const int L = p->L;
  // minibatch buffers: h[0] (inputs) and dh[0] (targets) of the gathered rows
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < n; ++i)
      if (perm[(size_t)ep * n + i] < 0 || perm[(size_t)ep * n + i] >= n) return QOC_EINVAL;
    MTRY(cudaMemcpyAsync(p->perm, perm + (size_t)ep * n, sizeof(int) * n, cudaMemcpyHostToDevice, p->stream));
    double acc = 0.0;
    int nbat = 0;
    std::vector<float> lbuf;
    for (int s = 0; s < n; s += batch) {
      const int B = (n - s) < batch ? (n - s) : batch;
      MTRY(mlp_gather(p->X, p->perm + s, B, p->d[0], p->h[0], p->stream));
      MTRY(mlp_gather(p->T, p->perm + s, B, p->d[L], p->dh[0], p->stream));
      qoc_status st = forward(p, p->h[0], B, 0);
      if (st != QOC_OK) return st;
      // targets sit in dh[0]; backward overwrites dh[k >= 1] only
      st = backward(p, p->h[0], p->dh[0], B);
      if (st != QOC_OK) return st;
      ++p->adam_t;
      const float c1 = 1.0f - powf(0.9f, (float)p->adam_t), c2 = 1.0f - powf(0.999f, (float)p->adam_t);
      MTRY(mlp_adam(p->w, p->g, p->m, p->v, (int)p->np, lr, 0.9f, 0.999f, 1e-8f, c1, c2, p->stream));
      MTRY(cudaMemcpyAsync(p->hbuf + (nbat % 64), p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
      ++nbat;
      if (nbat % 64 == 0) {
        MTRY(cudaStreamSynchronize(p->stream));
        for (int k = 0; k < 64; ++k) acc += p->hbuf[k];
      }
    }
    MTRY(cudaStreamSynchronize(p->stream));
    for (int k = 0; k < nbat % 64; ++k) acc += p->hbuf[k];
    losses[ep] = (float)(acc / nbat);
  }
  p->bf_valid = 0;
  return QOC_OK;
}

qoc_status qoc_mlp_gradient(qoc_mlp* p, const float* X, const float* T, int batch, float* loss,
                            float* grad) {
  if (!p || !X || !T || !loss || !grad || batch < 1 || batch > p->max_batch) return QOC_EINVAL;
  const int L = p->L;
  MTRY(cudaMemcpyAsync(p->h[0], X, sizeof(float) * (size_t)batch * p->d[0], cudaMemcpyHostToDevice, p->stream));
  MTRY(cudaMemcpyAsync(p->dh[0], T, sizeof(float) * (size_t)batch * p->d[L], cudaMemcpyHostToDevice, p->stream));
  qoc_status st = forward(p, p->h[0], batch, 0);
  if (st != QOC_OK) return st;
  st = backward(p, p->h[0], p->dh[0], batch);
  if (st != QOC_OK) return st;
  MTRY(cudaMemcpyAsync(grad, p->g, sizeof(float) * p->np, cudaMemcpyDeviceToHost, p->stream));
  MTRY(cudaMemcpyAsync(loss, p->loss, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
  return cu(cudaStreamSynchronize(p->stream));
}

qoc_status qoc_mlp_predict(qoc_mlp* p, const float* X, int n, float* Y, int bf16) {
  if (!p || !X || !Y || n < 1) return QOC_EINVAL;
  const int L = p->L;
  if (bf16 && !p->bf_valid) {
    MTRY(mlp_to_bf16(p->w, p->wbf, (int)p->np, p->stream));
    p->bf_valid = 1;
  }
  for (int s = 0; s < n; s += p->max_batch) {
    const int B = (n - s) < p->max_batch ? (n - s) : p->max_batch;
    MTRY(cudaMemcpyAsync(p->h[0], X + (size_t)s * p->d[0], sizeof(float) * (size_t)B * p->d[0],
                         cudaMemcpyHostToDevice, p->stream));
    qoc_status st = forward(p, p->h[0], B, bf16);
    if (st != QOC_OK) return st;
    MTRY(cudaMemcpyAsync(Y + (size_t)s * p->d[L], p->h[L], sizeof(float) * (size_t)B * p->d[L],
                         cudaMemcpyDeviceToHost, p->stream));
  }
  return cu(cudaStreamSynchronize(p->stream));
}

}  // extern "C"
