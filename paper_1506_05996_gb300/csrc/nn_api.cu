// C ABI of the learned correction (include/sem.h, sem_net_*): network objects, training
// steps on the GPU, and the correction N(r) added to the preconditioner in flexible PCG.
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/sem.h"
#include "nn.h"
#include "handle.h"

struct sem_net_s {
  sem::NnWeights w;
  sem::NnWork ws;   // training work space, grown to the largest mesh seen
  int step = 0;
  std::vector<void*> allocs, ws_allocs;
};

namespace {

int fail(int code, const std::string& msg) { return sem::report_error(code, msg); }

#define CKN(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n, std::vector<void*>& list) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e == cudaSuccess) list.push_back(*p);
  return e;
}

void free_all(std::vector<void*>& list) {
  for (void* q : list) cudaFree(q);
  list.clear();
}

// Work space for a mesh of ne elements with p3 nodes each; training adds the gradients.
int ensure_work(sem::NnWork& ws, std::vector<void*>& list, int ne, int p3, bool train) {
  if (ws.ne >= ne && ws.p3 >= p3 && (ws.train || !train) && ws.x0 != nullptr) return SEM_OK;
  free_all(list);
  ws = sem::NnWork();
  ws.ne = ne;
  ws.p3 = p3;
  ws.train = train;
  const size_t L = (size_t)ne * p3;
  CKN(dalloc(&ws.x0, L * sem::kNnIn, list));
  CKN(dalloc(&ws.a1, L * sem::kNnHid, list));
  CKN(dalloc(&ws.a2, L * sem::kNnHid, list));
  CKN(dalloc(&ws.y, L, list));
  CKN(dalloc(&ws.sigma, (size_t)ne, list));
  if (train) {
    CKN(dalloc(&ws.g1, L * sem::kNnHid, list));
    CKN(dalloc(&ws.g2, L * sem::kNnHid, list));
    CKN(dalloc(&ws.g3, L, list));
    CKN(dalloc(&ws.partial, (size_t)ne * sem::kNnParams, list));
    CKN(dalloc(&ws.grad, (size_t)sem::kNnParams, list));
    CKN(dalloc(&ws.eloss, (size_t)ne, list));
    CKN(dalloc(&ws.loss, 1, list));
    CKN(dalloc(&ws.c, L, list));   // G <= ne p^3
    CKN(dalloc(&ws.q, L, list));
    CKN(dalloc(&ws.dots, (size_t)(2 * sem::kNnMaxVecBlocks), list));
    CKN(dalloc(&ws.coef, 2, list));
  }
  return SEM_OK;
}

int check_vecs(sem_t* h, const void* a, const void* b) {
  if (h == nullptr || a == nullptr || b == nullptr || a == b) return fail(SEM_ERR_ARG, "bad handle or vectors");
  return SEM_OK;
}

}  // namespace

namespace sem {

int learned_attach(sem_t* h, sem_net_t* net) {
  h->net = net;
  h->invalidate();
  if (net == nullptr) return SEM_OK;
  const int p3 = h->d.p * h->d.p * h->d.p;
  if (int rc = ensure_work(h->nnws, h->nn_allocs, h->d.ne, p3, false)) return rc;
  // solver vectors live as long as the handle (h->allocs); the work space may be regrown
  if (h->d.nncorr == nullptr) CKN(dalloc(&h->d.nncorr, (size_t)h->nb.G, h->allocs));
  if (h->d.nns == nullptr) CKN(dalloc(&h->d.nns, (size_t)h->nb.G, h->allocs));
  if (h->d.rprev == nullptr) CKN(dalloc(&h->d.rprev, (size_t)h->nb.G, h->allocs));
  if (h->d.st_nn == nullptr) CKN(dalloc(&h->d.st_nn, 1, h->allocs));
  return SEM_OK;
}

cudaError_t learned_correction(sem_t* h, const double* r, const PcgState* st, cudaStream_t s) {
  cudaError_t e = nn_forward(h->d, h->net->w, h->nnws, r, h->mN, st, s);
  if (e == cudaSuccess) e = nn_gather(h->d, h->nnws, h->d.nncorr, st, s);
  return e;
}

}  // namespace sem

extern "C" {

int sem_net_create(uint64_t seed, sem_net_t** out) {
  if (out == nullptr) return fail(SEM_ERR_ARG, "out is NULL");
  *out = nullptr;
  sem_net_t* net = new sem_net_t();
  auto bail = [&](int rc) { sem_net_destroy(net); return rc; };
  std::vector<float> w(sem::kNnParams, 0.0f);
  std::mt19937_64 rng(seed);
  auto he = [&](int off, int n, int fan_in) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan_in));
    for (int q = 0; q < n; ++q) w[off + q] = (float)nd(rng);
  };
  he(sem::kOffW1, sem::kNnHid * sem::kNnIn * 27, sem::kNnIn * 27);
  he(sem::kOffW2, sem::kNnHid * sem::kNnHid * 27, sem::kNnHid * 27);
  // the last layer starts at zero: an untrained network adds nothing
  auto mk = [&](auto** p, size_t n) { return dalloc(p, n, net->allocs); };
  if (mk(&net->w.master, sem::kNnParams) || mk(&net->w.m, sem::kNnParams) || mk(&net->w.v, sem::kNnParams) ||
      mk(&net->w.w16, sem::kNnParams))
    return bail(fail(SEM_ERR_OOM, "cudaMalloc failed"));
  if (cudaMemcpy(net->w.master, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->w.m, 0, sizeof(float) * sem::kNnParams) != cudaSuccess ||
      cudaMemset(net->w.v, 0, sizeof(float) * sem::kNnParams) != cudaSuccess ||
      sem::nn_refresh_bf16(net->w, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return bail(fail(SEM_ERR_CUDA, "network initialisation failed"));
  *out = net;
  return SEM_OK;
}

void sem_net_destroy(sem_net_t* net) {
  if (net == nullptr) return;
  cudaDeviceSynchronize();
  free_all(net->ws_allocs);
  free_all(net->allocs);
  delete net;
}

int sem_net_num_params(void) { return sem::kNnParams; }

int sem_net_get_params(const sem_net_t* net, float* params_host, int n) {
  if (net == nullptr || params_host == nullptr || n != sem::kNnParams) return fail(SEM_ERR_ARG, "bad arguments");
  CKN(cudaMemcpy(params_host, net->w.master, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return SEM_OK;
}

int sem_net_set_params(sem_net_t* net, const float* params_host, int n) {
  if (net == nullptr || params_host == nullptr || n != sem::kNnParams) return fail(SEM_ERR_ARG, "bad arguments");
  CKN(cudaMemcpy(net->w.master, params_host, sizeof(float) * n, cudaMemcpyHostToDevice));
  CKN(cudaMemset(net->w.m, 0, sizeof(float) * n));
  CKN(cudaMemset(net->w.v, 0, sizeof(float) * n));
  net->step = 0;
  CKN(sem::nn_refresh_bf16(net->w, nullptr));
  CKN(cudaDeviceSynchronize());
  return SEM_OK;
}

int sem_net_gradient(sem_net_t* net, sem_t* h, const double* v_dev, const double* target_dev,
                     const double* r_dev, const double* z0_dev, int loss_kind, float* grad_host, double* loss_host) {
  if (net == nullptr) return fail(SEM_ERR_ARG, "NULL network");
  if (int rc = check_vecs(h, v_dev, target_dev)) return rc;
  if (loss_kind != SEM_NET_LOSS_L2 && loss_kind != SEM_NET_LOSS_ENERGY && loss_kind != SEM_NET_LOSS_ANGLE)
    return fail(SEM_ERR_ARG, "unknown loss");
  if (loss_kind == SEM_NET_LOSS_ANGLE && (r_dev == nullptr || z0_dev == nullptr))
    return fail(SEM_ERR_ARG, "the angle loss needs r and z0");
  const int p3 = h->d.p * h->d.p * h->d.p;
  if (int rc = ensure_work(net->ws, net->ws_allocs, h->d.ne, p3, true)) return rc;
  const sem::DevProblem& d = h->d;
  const sem::NnWork& ws = net->ws;
  cudaStream_t s = h->stream;
  CKN(sem::nn_forward(d, net->w, ws, v_dev, h->mN, nullptr, s));
  if (loss_kind == SEM_NET_LOSS_L2) {
    CKN(sem::nn_loss_l2(d, ws, target_dev, s));
  } else {
    // c = N(v), q = v - A c (the handle's operator precision), then the loss and dL/dy
    CKN(sem::nn_gather(d, ws, ws.c, nullptr, s));
    if (d.fp32) {
      float* wl = reinterpret_cast<float*>(d.wl);
      CKN(sem::launch_ax_local_f32(d, ws.c, wl, nullptr, s));
      CKN(sem::launch_residual_of_f32(d, wl, v_dev, ws.q, nullptr, s));
    } else {
      CKN(sem::launch_ax_local(d, ws.c, d.wl, nullptr, s));
      CKN(sem::launch_residual_of(d, d.wl, v_dev, ws.q, nullptr, s));
    }
    if (loss_kind == SEM_NET_LOSS_ENERGY)
      CKN(sem::nn_loss_energy(d, ws, v_dev, target_dev, s));
    else
      CKN(sem::nn_loss_angle(d, ws, r_dev, z0_dev, target_dev, s));
  }
  CKN(sem::nn_backward(d, net->w, ws, s));
  if (grad_host) CKN(cudaMemcpyAsync(grad_host, ws.grad, sizeof(float) * sem::kNnParams, cudaMemcpyDeviceToHost, s));
  double loss = 0.0;
  CKN(cudaMemcpyAsync(&loss, ws.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKN(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = loss;
  return SEM_OK;
}

int sem_net_train_step(sem_net_t* net, sem_t* h, const double* v_dev, const double* target_dev,
                       const double* r_dev, const double* z0_dev, int loss_kind, float lr, double* loss_host) {
  if (int rc = sem_net_gradient(net, h, v_dev, target_dev, r_dev, z0_dev, loss_kind, nullptr, loss_host)) return rc;
  net->step += 1;
  CKN(sem::nn_adam(net->w, net->ws, lr, net->step, h->stream));
  CKN(cudaStreamSynchronize(h->stream));
  return SEM_OK;
}

int sem_net_apply(sem_net_t* net, sem_t* h, const double* r_dev, double* out_dev) {
  if (net == nullptr) return fail(SEM_ERR_ARG, "NULL network");
  if (int rc = check_vecs(h, r_dev, out_dev)) return rc;
  const int p3 = h->d.p * h->d.p * h->d.p;
  if (int rc = ensure_work(net->ws, net->ws_allocs, h->d.ne, p3, net->ws.train)) return rc;
  CKN(sem::nn_forward(h->d, net->w, net->ws, r_dev, h->mN, nullptr, h->stream));
  CKN(sem::nn_gather(h->d, net->ws, out_dev, nullptr, h->stream));
  return SEM_OK;
}

int sem_set_learned(sem_t* h, sem_net_t* net, int stall_window, double stall_ratio, double accept_theta) {
  if (h == nullptr) return fail(SEM_ERR_ARG, "NULL handle");
  if (stall_window < 0 || stall_window > sem::kMaxStallWindow || !(stall_ratio > 0.0) || !std::isfinite(stall_ratio) ||
      std::isnan(accept_theta))
    return fail(SEM_ERR_ARG, "stall_window must be in 0..8, stall_ratio > 0 and accept_theta a number");
  CKN(cudaStreamSynchronize(h->stream));
  h->nn_window = stall_window;
  h->nn_ratio = stall_ratio;
  h->nn_theta = accept_theta;
  return sem::learned_attach(h, net);
}

int sem_learned_iterations(const sem_t* h, int* used_host) {
  if (h == nullptr || used_host == nullptr) return fail(SEM_ERR_ARG, "NULL argument");
  *used_host = (h->net != nullptr && h->st_host != nullptr) ? h->st_host->nn_used : 0;
  return SEM_OK;
}

}  // extern "C"
