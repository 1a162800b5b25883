// C ABI of the learned initialiser's set network: parameters, one training
// step (forward, Chamfer loss, backward, Adam) on the GPU kernels of
// km_setnet.cu, and prediction of starting centres from point samples.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/km.h"
#include "km_internal.cuh"

using namespace km;

struct km_setnet {
  int d = 0, k = 0, nparam = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  float *prm = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  long adam_t = 0;
  int capB = 0, capS = 0;
  float *xin = nullptr, *tin = nullptr;  // host inputs are copied here
  float *xs = nullptr, *ts = nullptr, *ms = nullptr, *w2t = nullptr, *h1 = nullptr, *h2 = nullptr;
  float *tile_pool = nullptr, *G = nullptr, *P = nullptr, *dG = nullptr, *loss = nullptr;
  float *dz2 = nullptr, *dz1 = nullptr, *part = nullptr;
  double* cout = nullptr;
  std::string err;
};

namespace {

km_status nfail(km_setnet* n, km_status s, const std::string& m) {
  n->err = m;
  return s;
}
#define KN_CUDA(n, call)                                                                           \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return nfail(n, e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA,                      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename T>
cudaError_t nalloc(T** p, size_t count) {
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

void free_work(km_setnet* n) {
  float* bufs[] = {n->xin, n->tin, n->xs, n->ts, n->ms, n->h1, n->h2, n->tile_pool, n->G, n->P, n->dG, n->dz2,
                   n->dz1, n->part};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (n->cout) cudaFree(n->cout);
  n->xin = n->tin = n->xs = n->ts = n->ms = n->h1 = n->h2 = n->tile_pool = n->G = n->P = n->dG = n->dz2 = n->dz1 =
      n->part = nullptr;
  n->cout = nullptr;
  n->capB = n->capS = 0;
}

km_status ensure(km_setnet* n, int B, int S) {
  if (B <= n->capB && S <= n->capS) return KM_OK;
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  free_work(n);
  const int64_t Pn = (int64_t)B * S;
  const int d = n->d, KD = n->k * n->d;
  KN_CUDA(n, nalloc(&n->xin, (size_t)Pn * d));
  KN_CUDA(n, nalloc(&n->tin, (size_t)B * KD));
  KN_CUDA(n, nalloc(&n->xs, (size_t)Pn * d));
  KN_CUDA(n, nalloc(&n->ts, (size_t)B * KD));
  KN_CUDA(n, nalloc(&n->ms, (size_t)B * 2 * d));
  KN_CUDA(n, nalloc(&n->h1, (size_t)Pn * kSetH));
  KN_CUDA(n, nalloc(&n->h2, (size_t)Pn * kSetH));
  KN_CUDA(n, nalloc(&n->tile_pool, (size_t)(Pn / 64) * kSetH));
  KN_CUDA(n, nalloc(&n->G, (size_t)B * kSetH));
  KN_CUDA(n, nalloc(&n->P, (size_t)B * KD));
  KN_CUDA(n, nalloc(&n->dG, (size_t)B * kSetH));
  KN_CUDA(n, nalloc(&n->dz2, (size_t)Pn * kSetH));
  KN_CUDA(n, nalloc(&n->dz1, (size_t)Pn * kSetH));
  KN_CUDA(n, nalloc(&n->part, (size_t)setnet_part_floats(Pn, d)));
  KN_CUDA(n, nalloc(&n->cout, (size_t)B * KD));
  n->capB = B;
  n->capS = S;
  return KM_OK;
}

SetNetArgs args(km_setnet* n, const float* x, const float* t, int B, int S) {
  SetNetArgs a{};
  a.x = x; a.t = t; a.B = B; a.S = S; a.d = n->d; a.k = n->k;
  a.prm = n->prm; a.grads = n->grads;
  a.xs = n->xs; a.ts = n->ts; a.ms = n->ms; a.w2t = n->w2t; a.h1 = n->h1; a.h2 = n->h2;
  a.tile_pool = n->tile_pool; a.G = n->G; a.P = n->P; a.dG = n->dG; a.loss = n->loss;
  a.dz2 = n->dz2; a.dz1 = n->dz1; a.part = n->part;
  return a;
}

// Points (and targets) on the device: copied from the host, or used as given.
km_status inputs(km_setnet* n, const float* x, const float* t, int B, int S, int mem, const float** xd,
                 const float** td) {
  if (B < 1 || S < 64 || S % 64) return nfail(n, KM_EINVAL, "need B >= 1 and S a positive multiple of 64");
  km_status s = ensure(n, B, S);
  if (s != KM_OK) return s;
  if (mem == KM_HOST) {
    KN_CUDA(n, cudaMemcpyAsync(n->xin, x, sizeof(float) * (size_t)B * S * n->d, cudaMemcpyHostToDevice, n->st));
    if (t) KN_CUDA(n, cudaMemcpyAsync(n->tin, t, sizeof(float) * (size_t)B * n->k * n->d, cudaMemcpyHostToDevice, n->st));
    *xd = n->xin;
    *td = t ? n->tin : nullptr;
  } else if (mem == KM_DEVICE_COPY || mem == KM_DEVICE_BORROW) {
    *xd = x;
    *td = t;
  } else {
    return nfail(n, KM_EINVAL, "bad mem kind");
  }
  return KM_OK;
}

}  // namespace

template <typename T>
static km_status sets_rotate(const T* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, const double* R,
                             const double* center, int64_t center_stride, int32_t transpose, T* out, void* stream) {
  if (!x || !R || !out || B < 1 || S < 1 || d < 1 || d > 3 || set_stride < 0 || center_stride < 0) return KM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_sets_rotate<T>(x, set_stride, B, S, d, R, center, center_stride, transpose ? 1 : 0, out, st) !=
      cudaSuccess)
    return KM_ECUDA;
  return KM_OK;
}

extern "C" {

km_status km_setnet_create(km_setnet** out, int32_t d, int32_t k, void* stream) {
  if (!out) return KM_EINVAL;
  *out = nullptr;
  km_setnet* n = new (std::nothrow) km_setnet();
  if (!n) return KM_ENOMEM;
  *out = n;
  if (d < 1 || d > 3 || k < 1 || k > kBatchMaxK) return nfail(n, KM_EINVAL, "need d in 1..3 and K in 1..64");
  n->d = d;
  n->k = k;
  n->nparam = setnet_param_count(d, k);
  if (stream) {
    n->st = static_cast<cudaStream_t>(stream);
  } else {
    KN_CUDA(n, cudaStreamCreate(&n->st));
    n->own_stream = true;
  }
  KN_CUDA(n, nalloc(&n->prm, (size_t)n->nparam));
  KN_CUDA(n, nalloc(&n->grads, (size_t)n->nparam));
  KN_CUDA(n, nalloc(&n->m, (size_t)n->nparam));
  KN_CUDA(n, nalloc(&n->v, (size_t)n->nparam));
  KN_CUDA(n, nalloc(&n->w2t, (size_t)kSetH * kSetH));
  KN_CUDA(n, nalloc(&n->loss, 1));
  KN_CUDA(n, cudaMemsetAsync(n->prm, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaMemsetAsync(n->grads, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  return KM_OK;
}

int64_t km_setnet_param_count(const km_setnet* n) { return n ? n->nparam : -1; }

km_status km_setnet_set_params(km_setnet* n, const float* params) {
  if (!n || !params) return KM_EINVAL;
  KN_CUDA(n, cudaMemcpyAsync(n->prm, params, sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->st));
  KN_CUDA(n, cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparam, n->st));
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  n->adam_t = 0;
  return KM_OK;
}

km_status km_setnet_get_params(km_setnet* n, float* params_out) {
  if (!n || !params_out) return KM_EINVAL;
  KN_CUDA(n, cudaMemcpyAsync(params_out, n->prm, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->st));
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  return KM_OK;
}

km_status km_setnet_get_grads(km_setnet* n, float* grads_out) {
  if (!n || !grads_out) return KM_EINVAL;
  KN_CUDA(n, cudaMemcpyAsync(grads_out, n->grads, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->st));
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  return KM_OK;
}

km_status km_setnet_loss_grad(km_setnet* n, const float* x, const float* targets, int32_t B, int32_t S,
                              int32_t mem, float* loss_out) {
  if (!n || !x || !targets) return KM_EINVAL;
  const float *xd = nullptr, *td = nullptr;
  km_status s = inputs(n, x, targets, B, S, mem, &xd, &td);
  if (s != KM_OK) return s;
  SetNetArgs a = args(n, xd, td, B, S);
  KN_CUDA(n, launch_setnet_forward(a, true, n->st));
  KN_CUDA(n, launch_setnet_backward(a, n->st));
  if (loss_out) {
    KN_CUDA(n, cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
    KN_CUDA(n, cudaStreamSynchronize(n->st));
  }
  return KM_OK;
}

km_status km_setnet_adam(km_setnet* n, float lr, float beta1, float beta2, float eps) {
  if (!n) return KM_EINVAL;
  n->adam_t += 1;
  const double c1 = 1.0 - std::pow((double)beta1, (double)n->adam_t);
  const double c2 = 1.0 - std::pow((double)beta2, (double)n->adam_t);
  KN_CUDA(n, launch_setnet_adam(n->prm, n->grads, n->m, n->v, n->nparam, lr, beta1, beta2, eps, (float)c1,
                                (float)c2, n->st));
  return KM_OK;
}

km_status km_setnet_train_step(km_setnet* n, const float* x, const float* targets, int32_t B, int32_t S,
                               int32_t mem, float lr, float* loss_out) {
  km_status s = km_setnet_loss_grad(n, x, targets, B, S, mem, nullptr);
  if (s != KM_OK) return s;
  s = km_setnet_adam(n, lr, 0.9f, 0.999f, 1e-8f);
  if (s != KM_OK) return s;
  if (loss_out) {
    KN_CUDA(n, cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
    KN_CUDA(n, cudaStreamSynchronize(n->st));
  }
  return KM_OK;
}

km_status km_setnet_predict(km_setnet* n, const float* x, int32_t B, int32_t S, int32_t mem, double* centroids_out) {
  if (!n || !x || !centroids_out) return KM_EINVAL;
  const float *xd = nullptr, *td = nullptr;
  km_status s = inputs(n, x, nullptr, B, S, mem, &xd, &td);
  if (s != KM_OK) return s;
  SetNetArgs a = args(n, xd, nullptr, B, S);
  KN_CUDA(n, launch_setnet_forward(a, false, n->st));
  KN_CUDA(n, launch_setnet_destandardize(n->P, n->ms, B, n->d, n->k, n->cout, n->st));
  KN_CUDA(n, cudaMemcpyAsync(centroids_out, n->cout, sizeof(double) * (size_t)B * n->k * n->d, cudaMemcpyDefault,
                             n->st));
  KN_CUDA(n, cudaStreamSynchronize(n->st));
  return KM_OK;
}

km_status km_sets_mean(const float* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, double* means_out,
                       void* stream) {
  if (!x || !means_out || B < 1 || S < 1 || d < 1 || d > 3 || set_stride < 0) return KM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_sets_mean(x, set_stride, B, S, d, means_out, st) != cudaSuccess) return KM_ECUDA;
  return KM_OK;
}

km_status km_sets_rotate_f32(const float* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, const double* R,
                             const double* center, int64_t center_stride, int32_t transpose, float* out, void* stream) {
  return sets_rotate<float>(x, set_stride, B, S, d, R, center, center_stride, transpose, out, stream);
}

km_status km_sets_rotate_f64(const double* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, const double* R,
                             const double* center, int64_t center_stride, int32_t transpose, double* out,
                             void* stream) {
  return sets_rotate<double>(x, set_stride, B, S, d, R, center, center_stride, transpose, out, stream);
}

int32_t km_setnet_dims(const km_setnet* n, int32_t* k_out) {
  if (!n) return -1;
  if (k_out) *k_out = n->k;
  return n->d;
}

void* km_setnet_stream(const km_setnet* n) { return n ? (void*)n->st : nullptr; }

const char* km_setnet_last_error(const km_setnet* n) { return n ? n->err.c_str() : "null network"; }

void km_setnet_destroy(km_setnet* n) {
  if (!n) return;
  free_work(n);
  float* bufs[] = {n->prm, n->grads, n->m, n->v, n->w2t, n->loss};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (n->own_stream && n->st) cudaStreamDestroy(n->st);
  delete n;
}

}  // extern "C"
