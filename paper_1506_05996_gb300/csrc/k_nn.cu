// Kernels of the learned correction (not in the paper): a per-element network of three
// 3x3x3 convolutions (5 -> 8 -> 8 -> 1 channels, ReLU after the first two) on the
// element's GLL grid, BF16 weights, FP32 activations and accumulation.
//
//   features:  s_l = (r_N / m_N) hbar^2, sigma_e = sqrt(mean s^2), channels
//              (s / sigma, hx/hbar, hy/hbar, hz/hbar, lambda hbar^2 / (1 + lambda hbar^2))
//   output:    c_l = y_l sigma_e, averaged over the local copies of each DOF
//   training:  loss = mean (y - t / sigma)^2 over local nodes, backward through the three
//              convolutions, per-element weight gradients summed over elements in index
//              order (deterministic), Adam on FP32 master weights.
#include <cuda_bf16.h>

#include "kcommon.cuh"
#include "nn.h"

namespace sem {
namespace {

constexpr int kNnBlock = 256;

__device__ __forceinline__ bool net_skip(const PcgState* st) {
  return st != nullptr && (st->done != 0 || st->nn_off != 0);
}

__device__ __forceinline__ void node_ijk(int l, int p, int& i, int& j, int& k) {
  i = l % p;
  j = (l / p) % p;
  k = l / (p * p);
}

// one CTA per element
template <int p>
__global__ void __launch_bounds__(kNnBlock) nn_features_kernel(const DevProblem d, const double* __restrict__ r,
                                                               const double* __restrict__ mN, float* __restrict__ x,
                                                               double* __restrict__ sigma, const PcgState* st) {
  constexpr int p3 = p * p * p;
  if (net_skip(st)) return;
  const int e = blockIdx.x;
  const double hx = d.hbox[3 * e], hy = d.hbox[3 * e + 1], hz = d.hbox[3 * e + 2];
  const double hbar = (hx + hy + hz) / 3.0, h2 = hbar * hbar;
  double s2 = 0.0;
  float* xe = x + (size_t)e * kNnIn * p3;
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    const int g = d.l2g[(size_t)e * p3 + l];
    const double s = r[g] / mN[g] * h2;
    s2 += s * s;
  }
  __shared__ double ssig;
  const double tot = block_sum<kNnBlock>(s2);
  if (threadIdx.x == 0) ssig = sqrt(tot / p3) + 1e-300;
  __syncthreads();
  const double sg = ssig;
  const double q = d.lambda * h2;
  const float c1 = (float)(hx / hbar), c2 = (float)(hy / hbar), c3 = (float)(hz / hbar), c4 = (float)(q / (1.0 + q));
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    const int g = d.l2g[(size_t)e * p3 + l];
    xe[l] = (float)(r[g] / mN[g] * h2 / sg);
    xe[1 * p3 + l] = c1;
    xe[2 * p3 + l] = c2;
    xe[3 * p3 + l] = c3;
    xe[4 * p3 + l] = c4;
  }
  if (threadIdx.x == 0) sigma[e] = sg;
}

// y[co][l] = b[co] + sum_{ci, tap} W[co][ci][tap] x[ci][l + off(tap)] (zero outside), optional ReLU
template <int p, int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(kNnBlock) conv_fwd_kernel(const float* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                            const float* __restrict__ bias, float* __restrict__ out,
                                                            const PcgState* st) {
  constexpr int p3 = p * p * p;
  if (net_skip(st)) return;
  __shared__ float sx[CIN * p3];
  __shared__ float sw[COUT * CIN * 27];
  __shared__ float sb[COUT];
  const int e = blockIdx.x;
  const float* xe = in + (size_t)e * CIN * p3;
  for (int q = threadIdx.x; q < CIN * p3; q += kNnBlock) sx[q] = xe[q];
  for (int q = threadIdx.x; q < COUT * CIN * 27; q += kNnBlock) sw[q] = __bfloat162float(W[q]);
  if (threadIdx.x < COUT) sb[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  float* oe = out + (size_t)e * COUT * p3;
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    int i, j, k;
    node_ijk(l, p, i, j, k);
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = sb[co];
    for (int a = 0; a < 3; ++a) {
      const int ii = i + a - 1;
      if (ii < 0 || ii >= p) continue;
      for (int c = 0; c < 3; ++c) {
        const int jj = j + c - 1;
        if (jj < 0 || jj >= p) continue;
        for (int dd = 0; dd < 3; ++dd) {
          const int kk = k + dd - 1;
          if (kk < 0 || kk >= p) continue;
          const int tap = (a * 3 + c) * 3 + dd, ln = ii + p * (jj + p * kk);
#pragma unroll
          for (int ci = 0; ci < CIN; ++ci) {
            const float v = sx[ci * p3 + ln];
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] += sw[(co * CIN + ci) * 27 + tap] * v;
          }
        }
      }
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co) oe[co * p3 + l] = RELU ? fmaxf(acc[co], 0.0f) : acc[co];
  }
}

// gin[ci][l] = sum_{co, tap} W[co][ci][tap] gout[co][l - off(tap)], times (act_in > 0) if MASK
template <int p, int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(kNnBlock) conv_bwd_data_kernel(const float* __restrict__ gout,
                                                                 const __nv_bfloat16* __restrict__ W,
                                                                 const float* __restrict__ act_in,
                                                                 float* __restrict__ gin) {
  constexpr int p3 = p * p * p;
  __shared__ float sg[COUT * p3];
  __shared__ float sw[COUT * CIN * 27];
  const int e = blockIdx.x;
  const float* ge = gout + (size_t)e * COUT * p3;
  for (int q = threadIdx.x; q < COUT * p3; q += kNnBlock) sg[q] = ge[q];
  for (int q = threadIdx.x; q < COUT * CIN * 27; q += kNnBlock) sw[q] = __bfloat162float(W[q]);
  __syncthreads();
  float* gi = gin + (size_t)e * CIN * p3;
  const float* ai = act_in + (size_t)e * CIN * p3;
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    int i, j, k;
    node_ijk(l, p, i, j, k);
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
    for (int a = 0; a < 3; ++a) {
      const int ii = i - (a - 1);
      if (ii < 0 || ii >= p) continue;
      for (int c = 0; c < 3; ++c) {
        const int jj = j - (c - 1);
        if (jj < 0 || jj >= p) continue;
        for (int dd = 0; dd < 3; ++dd) {
          const int kk = k - (dd - 1);
          if (kk < 0 || kk >= p) continue;
          const int tap = (a * 3 + c) * 3 + dd, lo = ii + p * (jj + p * kk);
#pragma unroll
          for (int co = 0; co < COUT; ++co) {
            const float gv = sg[co * p3 + lo];
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) acc[ci] += sw[(co * CIN + ci) * 27 + tap] * gv;
          }
        }
      }
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) gi[ci * p3 + l] = (MASK && !(ai[ci * p3 + l] > 0.0f)) ? 0.0f : acc[ci];
  }
}

// per element: gW[co][ci][tap] = sum_l gout[co][l] x[ci][l + off(tap)], gb[co] = sum_l gout[co][l]
template <int p, int CIN, int COUT>
__global__ void __launch_bounds__(kNnBlock) conv_bwd_weight_kernel(const float* __restrict__ gout,
                                                                   const float* __restrict__ in,
                                                                   float* __restrict__ partial, int stride,
                                                                   int offset) {
  constexpr int p3 = p * p * p, NW = COUT * CIN * 27;
  __shared__ float sg[COUT * p3];
  __shared__ float sx[CIN * p3];
  const int e = blockIdx.x;
  for (int q = threadIdx.x; q < COUT * p3; q += kNnBlock) sg[q] = gout[(size_t)e * COUT * p3 + q];
  for (int q = threadIdx.x; q < CIN * p3; q += kNnBlock) sx[q] = in[(size_t)e * CIN * p3 + q];
  __syncthreads();
  float* pe = partial + (size_t)e * stride + offset;
  for (int w = threadIdx.x; w < NW + COUT; w += kNnBlock) {
    float acc = 0.0f;
    if (w < NW) {
      const int tap = w % 27, ci = (w / 27) % CIN, co = w / (27 * CIN);
      const int da = tap / 9 - 1, dc = (tap / 3) % 3 - 1, dd = tap % 3 - 1;
      for (int l = 0; l < p3; ++l) {
        int i, j, k;
        node_ijk(l, p, i, j, k);
        const int ii = i + da, jj = j + dc, kk = k + dd;
        if (ii < 0 || ii >= p || jj < 0 || jj >= p || kk < 0 || kk >= p) continue;
        acc += sg[co * p3 + l] * sx[ci * p3 + ii + p * (jj + p * kk)];
      }
    } else {
      const int co = w - NW;
      for (int l = 0; l < p3; ++l) acc += sg[co * p3 + l];
    }
    pe[w] = acc;
  }
}

// grad[j] = sum over elements of partial[e][j], elements in index order
__global__ void reduce_partials_kernel(int ne, int n, int stride, const float* __restrict__ partial,
                                       float* __restrict__ grad) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = 0; e < ne; ++e) s += partial[(size_t)e * stride + j];
    grad[j] = (float)s;
  }
}

// d = y - t / sigma at every local node; gout = 2 d / L; loss partial per element
template <int p>
__global__ void __launch_bounds__(kNnBlock) nn_loss_kernel(const DevProblem d, const float* __restrict__ y,
                                                           const double* __restrict__ sigma,
                                                           const double* __restrict__ target,
                                                           float* __restrict__ gout, double* __restrict__ eloss,
                                                           double invL) {
  constexpr int p3 = p * p * p;
  const int e = blockIdx.x;
  const double sg = sigma[e];
  double acc = 0.0;
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    const int g = d.l2g[(size_t)e * p3 + l];
    const double diff = (double)y[(size_t)e * p3 + l] - target[g] / sg;
    gout[(size_t)e * p3 + l] = (float)(2.0 * diff * invL);
    acc += diff * diff;
  }
  const double tot = block_sum<kNnBlock>(acc);
  if (threadIdx.x == 0) eloss[e] = tot;
}

// per block: sums of delta.v and c.(v + q) over the DOFs (partials [2][gridDim.x])
__global__ void __launch_bounds__(kVecBlock) nn_energy_dots_kernel(int G, const double* __restrict__ v,
                                                                   const double* __restrict__ delta,
                                                                   const double* __restrict__ c,
                                                                   const double* __restrict__ q,
                                                                   double* __restrict__ partial) {
  double a = 0.0, b = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    a += delta[g] * v[g];
    b += c[g] * (v[g] + q[g]);
  }
  const double sa = block_sum<kVecBlock>(a);
  const double sb = block_sum<kVecBlock>(b);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sa;
    partial[gridDim.x + blockIdx.x] = sb;
  }
}

// loss = 1 - c.(v + q) / delta.v; coef[0] = delta.v (partials summed in block order)
__global__ void nn_energy_finish_kernel(int nb, const double* __restrict__ partial, double* __restrict__ coef,
                                        double* __restrict__ loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += partial[i];
      b += partial[nb + i];
    }
    coef[0] = a;
    *loss = 1.0 - b / a;
  }
}

// energy: dL/dc = -2 q / delta.v, written over q
__global__ void nn_energy_dc_kernel(int G, const double* __restrict__ coef, double* __restrict__ q) {
  const double k = -2.0 / coef[0];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) q[g] *= k;
}

// per block: a = z.r, Q = z.(r - q) (= z^T A z), E = (delta + z0).r with z = z0 + c
__global__ void __launch_bounds__(kVecBlock) nn_angle_dots_kernel(int G, const double* __restrict__ r,
                                                                  const double* __restrict__ z0,
                                                                  const double* __restrict__ delta,
                                                                  const double* __restrict__ c,
                                                                  const double* __restrict__ q,
                                                                  double* __restrict__ partial) {
  double a = 0.0, Q = 0.0, E = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const double z = z0[g] + c[g], rg = r[g];
    a += z * rg;
    Q += z * (rg - q[g]);
    E += (delta[g] + z0[g]) * rg;
  }
  const double sa = block_sum<kVecBlock>(a);
  const double sQ = block_sum<kVecBlock>(Q);
  const double sE = block_sum<kVecBlock>(E);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sa;
    partial[gridDim.x + blockIdx.x] = sQ;
    partial[2 * gridDim.x + blockIdx.x] = sE;
  }
}

// loss = 1 - a / sqrt(Q E); coef = (-1 / sqrt(Q E), a / Q)
__global__ void nn_angle_finish_kernel(int nb, const double* __restrict__ partial, double* __restrict__ coef,
                                       double* __restrict__ loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double a = 0.0, Q = 0.0, E = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += partial[i];
      Q += partial[nb + i];
      E += partial[2 * nb + i];
    }
    const double rs = 1.0 / sqrt(Q * E);
    *loss = 1.0 - a * rs;
    coef[0] = -rs;
    coef[1] = a / Q;
  }
}

// angle: dL/dc = k1 (r - k2 A z) with A z = r - q, written over q (0 on masked DOFs: r, q are)
__global__ void nn_angle_dc_kernel(int G, const double* __restrict__ coef, const double* __restrict__ r,
                                   double* __restrict__ q) {
  const double k1 = coef[0], k2 = coef[1];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    q[g] = k1 * (r[g] - k2 * (r[g] - q[g]));
}

// dL/dy_l = dL/dc_N sigma_e / multiplicity_N, 0 on masked DOFs
template <int p>
__global__ void __launch_bounds__(kNnBlock) nn_dc_to_gout_kernel(const DevProblem d, const double* __restrict__ dc,
                                                                 const double* __restrict__ sigma,
                                                                 float* __restrict__ gout) {
  constexpr int p3 = p * p * p;
  const int e = blockIdx.x;
  const double sg = sigma[e];
  for (int l = threadIdx.x; l < p3; l += kNnBlock) {
    const int g = d.l2g[(size_t)e * p3 + l];
    const double mult = (double)(d.g2l_off[g + 1] - d.g2l_off[g]);
    gout[(size_t)e * p3 + l] = d.mask[g] ? 0.0f : (float)(dc[g] * sg / mult);
  }
}

__global__ void sum_in_order_kernel(int n, const double* __restrict__ v, double scale, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s * scale;
  }
}

__global__ void adam_kernel(int n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ w16, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const float gj = g[j];
    const float mj = b1 * m[j] + (1.0f - b1) * gj;
    const float vj = b2 * v[j] + (1.0f - b2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    const float wj = w[j] - lr * (mj / c1) / (sqrtf(vj / c2) + eps);
    w[j] = wj;
    w16[j] = __float2bfloat16_rn(wj);
  }
}

__global__ void to_bf16_kernel(int n, const float* __restrict__ w, __nv_bfloat16* __restrict__ w16) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    w16[j] = __float2bfloat16_rn(w[j]);
}

// global correction: c_N = mean over the local copies of y_l sigma_e; 0 on masked DOFs
__global__ void nn_gather_kernel(const DevProblem d, const float* __restrict__ y, const double* __restrict__ sigma,
                                 double* __restrict__ out, const PcgState* st) {
  if (net_skip(st)) return;
  const int p3 = d.p * d.p * d.p;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < d.G; g += gridDim.x * blockDim.x) {
    double s = 0.0;
    const int q0 = d.g2l_off[g], q1 = d.g2l_off[g + 1];
    if (!d.mask[g]) {
      for (int q = q0; q < q1; ++q) {
        const int l = d.g2l_idx[q];
        s += (double)y[l] * sigma[l / p3];
      }
      s /= (double)(q1 - q0);
    }
    out[g] = s;
  }
}

template <int p>
cudaError_t forward_p(const DevProblem& d, const NnWeights& w, const NnWork& ws, const double* r, const double* mN,
                      const PcgState* st, cudaStream_t s) {
  nn_features_kernel<p><<<d.ne, kNnBlock, 0, s>>>(d, r, mN, ws.x0, ws.sigma, st);
  conv_fwd_kernel<p, kNnIn, kNnHid, true><<<d.ne, kNnBlock, 0, s>>>(ws.x0, w.w16 + kOffW1, w.master + kOffB1, ws.a1,
                                                                     st);
  conv_fwd_kernel<p, kNnHid, kNnHid, true><<<d.ne, kNnBlock, 0, s>>>(ws.a1, w.w16 + kOffW2, w.master + kOffB2,
                                                                      ws.a2, st);
  conv_fwd_kernel<p, kNnHid, 1, false><<<d.ne, kNnBlock, 0, s>>>(ws.a2, w.w16 + kOffW3, w.master + kOffB3,
                                                                  ws.y, st);
  for (int q = 0; q < 4; ++q) count_launch();
  return cudaGetLastError();
}

template <int p>
cudaError_t loss_l2_p(const DevProblem& d, const NnWork& ws, const double* target, double invL, cudaStream_t s) {
  nn_loss_kernel<p><<<d.ne, kNnBlock, 0, s>>>(d, ws.y, ws.sigma, target, ws.g3, ws.eloss, invL);
  sum_in_order_kernel<<<1, 32, 0, s>>>(d.ne, ws.eloss, invL, ws.loss);
  count_launch();
  count_launch();
  return cudaGetLastError();
}

template <int p>
cudaError_t dc_to_gout_p(const DevProblem& d, const NnWork& ws, cudaStream_t s) {
  nn_dc_to_gout_kernel<p><<<d.ne, kNnBlock, 0, s>>>(d, ws.q, ws.sigma, ws.g3);
  count_launch();
  return cudaGetLastError();
}

template <int p>
cudaError_t backward_p(const DevProblem& d, const NnWeights& w, const NnWork& ws, cudaStream_t s) {
  // layer 3 (8 -> 1): weights, then data into layer-2 activations (masked by ReLU)
  conv_bwd_weight_kernel<p, kNnHid, 1><<<d.ne, kNnBlock, 0, s>>>(ws.g3, ws.a2, ws.partial, kNnParams, kOffW3);
  conv_bwd_data_kernel<p, kNnHid, 1, true><<<d.ne, kNnBlock, 0, s>>>(ws.g3, w.w16 + kOffW3, ws.a2, ws.g2);
  // layer 2 (8 -> 8)
  conv_bwd_weight_kernel<p, kNnHid, kNnHid><<<d.ne, kNnBlock, 0, s>>>(ws.g2, ws.a1, ws.partial, kNnParams, kOffW2);
  conv_bwd_data_kernel<p, kNnHid, kNnHid, true><<<d.ne, kNnBlock, 0, s>>>(ws.g2, w.w16 + kOffW2, ws.a1, ws.g1);
  // layer 1 (5 -> 8): weights only
  conv_bwd_weight_kernel<p, kNnIn, kNnHid><<<d.ne, kNnBlock, 0, s>>>(ws.g1, ws.x0, ws.partial, kNnParams, kOffW1);
  reduce_partials_kernel<<<(kNnParams + 255) / 256, 256, 0, s>>>(d.ne, kNnParams, kNnParams, ws.partial, ws.grad);
  for (int q = 0; q < 6; ++q) count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t nn_forward(const DevProblem& d, const NnWeights& w, const NnWork& ws, const double* r, const double* mN,
                       const PcgState* st, cudaStream_t s) {
  switch (d.p) {
    case 3: return forward_p<3>(d, w, ws, r, mN, st, s);
    case 4: return forward_p<4>(d, w, ws, r, mN, st, s);
    case 5: return forward_p<5>(d, w, ws, r, mN, st, s);
    case 6: return forward_p<6>(d, w, ws, r, mN, st, s);
    case 7: return forward_p<7>(d, w, ws, r, mN, st, s);
    case 8: return forward_p<8>(d, w, ws, r, mN, st, s);
    case 9: return forward_p<9>(d, w, ws, r, mN, st, s);
    default: return cudaErrorInvalidValue;
  }
}

#define NN_DISPATCH_P(call)           \
  switch (d.p) {                      \
    case 3: { constexpr int P_ = 3; return call; } \
    case 4: { constexpr int P_ = 4; return call; } \
    case 5: { constexpr int P_ = 5; return call; } \
    case 6: { constexpr int P_ = 6; return call; } \
    case 7: { constexpr int P_ = 7; return call; } \
    case 8: { constexpr int P_ = 8; return call; } \
    case 9: { constexpr int P_ = 9; return call; } \
    default: return cudaErrorInvalidValue;          \
  }

cudaError_t nn_loss_l2(const DevProblem& d, const NnWork& ws, const double* target, cudaStream_t s) {
  const double invL = 1.0 / ((double)d.ne * d.p * d.p * d.p);
  NN_DISPATCH_P(loss_l2_p<P_>(d, ws, target, invL, s))
}

cudaError_t nn_loss_energy(const DevProblem& d, const NnWork& ws, const double* v, const double* delta,
                           cudaStream_t s) {
  if (d.nblk > kNnMaxVecBlocks) return cudaErrorInvalidValue;
  nn_energy_dots_kernel<<<d.nblk, kVecBlock, 0, s>>>(d.G, v, delta, ws.c, ws.q, ws.dots);
  nn_energy_finish_kernel<<<1, 32, 0, s>>>(d.nblk, ws.dots, ws.coef, ws.loss);
  nn_energy_dc_kernel<<<d.nblk, kVecBlock, 0, s>>>(d.G, ws.coef, ws.q);
  for (int q = 0; q < 3; ++q) count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  NN_DISPATCH_P(dc_to_gout_p<P_>(d, ws, s))
}

cudaError_t nn_loss_angle(const DevProblem& d, const NnWork& ws, const double* r, const double* z0,
                          const double* delta, cudaStream_t s) {
  if (d.nblk > kNnMaxVecBlocks) return cudaErrorInvalidValue;
  nn_angle_dots_kernel<<<d.nblk, kVecBlock, 0, s>>>(d.G, r, z0, delta, ws.c, ws.q, ws.dots);
  nn_angle_finish_kernel<<<1, 32, 0, s>>>(d.nblk, ws.dots, ws.coef, ws.loss);
  nn_angle_dc_kernel<<<d.nblk, kVecBlock, 0, s>>>(d.G, ws.coef, r, ws.q);
  for (int q = 0; q < 3; ++q) count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  NN_DISPATCH_P(dc_to_gout_p<P_>(d, ws, s))
}

cudaError_t nn_backward(const DevProblem& d, const NnWeights& w, const NnWork& ws, cudaStream_t s) {
  NN_DISPATCH_P(backward_p<P_>(d, w, ws, s))
}

cudaError_t nn_gather(const DevProblem& d, const NnWork& ws, double* out, const PcgState* st, cudaStream_t s) {
  nn_gather_kernel<<<d.nblk, kVecBlock, 0, s>>>(d, ws.y, ws.sigma, out, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t nn_adam(NnWeights& w, const NnWork& ws, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<(kNnParams + 255) / 256, 256, 0, s>>>(kNnParams, w.master, w.m, w.v, ws.grad, w.w16, lr, b1, b2, eps,
                                                      c1, c2);
  count_launch();
  return cudaGetLastError();
}

cudaError_t nn_refresh_bf16(NnWeights& w, cudaStream_t s) {
  to_bf16_kernel<<<(kNnParams + 255) / 256, 256, 0, s>>>(kNnParams, w.master, w.w16);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sem
