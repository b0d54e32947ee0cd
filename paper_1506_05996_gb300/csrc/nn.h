// Learned correction network (not in the paper): parameter layout, device buffers and
// launchers (k_nn.cu). The flat parameter vector is [W1, b1, W2, b2, W3, b3] with
// W[co][ci][a][c][d] for the tap (a, c, d) of the 3x3x3 correlation along (i, j, k).
#pragma once

#include <cuda_bf16.h>

#include "device.h"

namespace sem {

constexpr int kNnIn = 5, kNnHid = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kNnHid * kNnIn * 27;
constexpr int kOffW2 = kOffB1 + kNnHid, kOffB2 = kOffW2 + kNnHid * kNnHid * 27;
constexpr int kOffW3 = kOffB2 + kNnHid, kOffB3 = kOffW3 + kNnHid * 27;
constexpr int kNnParams = kOffB3 + 1;   // 3041

struct NnWeights {
  float* master = nullptr;            // FP32 master weights and biases [kNnParams]
  float *m = nullptr, *v = nullptr;   // Adam moments
  __nv_bfloat16* w16 = nullptr;       // BF16 copy used by the kernels (weights part)
};

// Work space for one mesh size (ne elements of p^3 nodes).
struct NnWork {
  int ne = 0, p3 = 0;
  bool train = false;
  float *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *y = nullptr;
  double* sigma = nullptr;            // per-element scale sigma_e
  float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *partial = nullptr, *grad = nullptr;
  double *eloss = nullptr, *loss = nullptr;
  // energy / angle losses: global correction c, q = v - A c (then dL/dc in place), block
  // partials and the loss coefficients
  double *c = nullptr, *q = nullptr, *dots = nullptr, *coef = nullptr;
};

constexpr int kNnMaxVecBlocks = 2048;   // >= DevProblem::nblk (partials of the energy dots)

enum NnLoss { NN_LOSS_L2 = 0, NN_LOSS_ENERGY = 1, NN_LOSS_ANGLE = 2 };

// features + the three convolutions: ws.y (local outputs) and ws.sigma; with st (inside
// flexible PCG) the kernels do nothing once the solve stopped or st->nn_off is set
cudaError_t nn_forward(const DevProblem& d, const NnWeights& w, const NnWork& ws, const double* r, const double* mN,
                       const PcgState* st, cudaStream_t s);
// L2 loss against the global target (sampled at the local nodes): *ws.loss and ws.g3 = dL/dy
cudaError_t nn_loss_l2(const DevProblem& d, const NnWork& ws, const double* target, cudaStream_t s);
// energy loss, given ws.c = N(v) and ws.q = mask ? 0 : v - A c: *ws.loss and ws.g3 = dL/dy
cudaError_t nn_loss_energy(const DevProblem& d, const NnWork& ws, const double* v, const double* delta,
                           cudaStream_t s);
// angle loss of z = z0 + c against e = delta + z0 (A e = r), given ws.c and ws.q as above
cudaError_t nn_loss_angle(const DevProblem& d, const NnWork& ws, const double* r, const double* z0,
                          const double* delta, cudaStream_t s);
// backward through the three convolutions from ws.g3: ws.grad
cudaError_t nn_backward(const DevProblem& d, const NnWeights& w, const NnWork& ws, cudaStream_t s);
// global correction from ws.y, ws.sigma (average over local copies, 0 on masked DOFs)
cudaError_t nn_gather(const DevProblem& d, const NnWork& ws, double* out, const PcgState* st, cudaStream_t s);
cudaError_t nn_adam(NnWeights& w, const NnWork& ws, float lr, int step, cudaStream_t s);
cudaError_t nn_refresh_bf16(NnWeights& w, cudaStream_t s);

}  // namespace sem
