// Device helpers shared by the kernel translation units (kernels.cu, k_ax*.cu, k_sw*.cu).
#pragma once

#include <cmath>

#include "device.h"

namespace sem {

void count_launch();   // adds one to kernel_launch_count() of this thread

namespace {

__device__ __forceinline__ bool stopped(const PcgState* st) { return st != nullptr && st->done != 0; }

// The state of the right-hand side this CTA works on in a block solve (blockIdx.y; the
// first and only one otherwise), or null outside a solve.
__device__ __forceinline__ const PcgState* st_rhs(const PcgState* st) {
  return st != nullptr ? st + blockIdx.y : nullptr;
}

// Mixed path: replace the recursive residual by b - A u (FP64 operator) whenever it has
// dropped by this factor since the last replacement, and before accepting convergence.
constexpr double kReplaceFactor = 1e-3;

// Sum over a block of BS threads; the result is valid in warp 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  static_assert(BS % 32 == 0 && BS <= 1024, "block size");
  __shared__ double sh[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < BS / 32) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// Grid reduction: every block writes its partial; the last block to arrive sums the
// partials in index order. Returns true in all threads of that last block, where
// `total` is valid in thread 0.
template <int BS>
__device__ __forceinline__ bool grid_reduce(double v, double* partial, unsigned int* counter, double& total) {
  __shared__ bool last;
  const double bs = block_sum<BS>(v);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += BS) s += __ldcg(&partial[i]);
  total = block_sum<BS>(s);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// NV sums at once (partial holds NV * gridDim.x entries): the same last-block rule;
// tot[] is valid in thread 0 of the last block.
template <int BS, int NV>
__device__ __forceinline__ bool grid_reduce_n(const double (&v)[NV], double* partial, unsigned int* counter,
                                              double (&tot)[NV]) {
  __shared__ bool last_n;
  double bsum[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) bsum[k] = block_sum<BS>(v[k]);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partial[k * gridDim.x + blockIdx.x] = bsum[k];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    last_n = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last_n) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += BS) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] += __ldcg(&partial[k * gridDim.x + i]);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = block_sum<BS>(s[k]);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// G = w |J| J^-1 J^-T (6 entries) and m = w |J| at reference point (a, b, c) from the
// 8 vertices xv[corner*3 + dim]. J[r][s] = d x_r / d xi_s of the trilinear map.
template <typename T>
__device__ __forceinline__ void geom_point(const T* xv, T a, T b, T c, T w, T G[6], T& m, T& det) {
  T J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const T one = 1, half = 0.5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const T sa = ((q == 1) | (q == 2) | (q == 5) | (q == 6)) ? one : -one;
    const T sb = ((q == 2) | (q == 3) | (q == 6) | (q == 7)) ? one : -one;
    const T sc = (q >= 4) ? one : -one;
    const T fa = half * (one + sa * a), fb = half * (one + sb * b), fc = half * (one + sc * c);
    const T d0 = half * sa * fb * fc, d1 = half * sb * fa * fc, d2 = half * sc * fa * fb;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T x = xv[3 * q + r];
      J[r][0] += x * d0;
      J[r][1] += x * d1;
      J[r][2] += x * d2;
    }
  }
  T C[3][3];
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  const T s = w / det;   // inv(J)[r][c] = C[c][r] / det
  G[0] = s * (C[0][0] * C[0][0] + C[1][0] * C[1][0] + C[2][0] * C[2][0]);
  G[1] = s * (C[0][0] * C[0][1] + C[1][0] * C[1][1] + C[2][0] * C[2][1]);
  G[2] = s * (C[0][0] * C[0][2] + C[1][0] * C[1][2] + C[2][0] * C[2][2]);
  G[3] = s * (C[0][1] * C[0][1] + C[1][1] * C[1][1] + C[2][1] * C[2][1]);
  G[4] = s * (C[0][1] * C[0][2] + C[1][1] * C[1][2] + C[2][1] * C[2][2]);
  G[5] = s * (C[0][2] * C[0][2] + C[1][2] * C[1][2] + C[2][2] * C[2][2]);
  m = w * det;
}

template <typename T> __device__ __forceinline__ const T* geo_of(const DevProblem& d);
template <> __device__ __forceinline__ const double* geo_of<double>(const DevProblem& d) { return d.geo; }
template <> __device__ __forceinline__ const float* geo_of<float>(const DevProblem& d) { return d.geo32; }
template <> __device__ __forceinline__ const __nv_bfloat16* geo_of<__nv_bfloat16>(const DevProblem& d) {
  return d.geo16;
}
// binary64 -> binary32, round to nearest (ties to even), written from the IEEE-754 bit
// layouts with 32-bit integer operations. On GB300 the conversion instruction runs on
// the FP64 pipe, at about 1/64 of the FP32 rate. The memory-bound PCG vector kernels that
// write FP32 copies of FP64 vectors use this instead (measured faster there); inside the
// arithmetic-heavy element kernels the instruction stays (this branchy form was measured
// slower there). Correctly rounded, so it gives the instruction's bits
// (sem_selfcheck_convert).
__device__ __forceinline__ float f64_to_f32(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned sign = hi & 0x80000000u, mh = hi & 0xfffffu;
  const int e64 = (int)((hi >> 20) & 0x7ffu);
  if (e64 == 0x7ff)   // infinity, or NaN (kept quiet)
    return __uint_as_float(sign | 0x7f800000u | (((mh | lo) != 0u) ? (0x400000u | (mh << 3) | (lo >> 29)) : 0u));
  const int e = e64 - 1023 + 127;   // biased binary32 exponent
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  if (e >= 1) {
    // 23 kept fraction bits, 29 dropped; a carry out of the fraction steps the exponent
    // (up to infinity), as rounding requires
    const unsigned m = (mh << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((sign | ((unsigned)e << 23) | m) + up);
  }
  if (e64 == 0) return __uint_as_float(sign);   // zero or binary64 subnormal: rounds to zero
  // binary32 subnormal or zero: q = round((2^52 + fraction) / 2^sh) units of 2^-149
  const int sh = 52 - (e64 - 1023 + 149);       // at least 30 here
  if (sh > 53) return __uint_as_float(sign);    // below half the smallest subnormal
  const unsigned long long M = ((unsigned long long)(mh | 0x100000u) << 32) | lo;
  const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  const unsigned long long up = (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(sign | (unsigned)(q + up));
}

// A stored factor as the kernel's arithmetic type.
template <typename T> __device__ __forceinline__ T factor(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T factor(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T factor(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

// Local index of element-interior DOF g < d.Gi: the numbering puts the (n-1)^3 interior
// nodes of each element first, element by element, in local order.
__device__ __forceinline__ int interior_local(const DevProblem& d, int g) {
  const int p = d.p, m = p - 2, m3 = m * m * m;
  const int e = g / m3;
  int r = g - e * m3;
  const int a = r % m;
  r /= m;
  const int b = r % m, c = r / m;
  return e * p * p * p + (a + 1) + p * ((b + 1) + p * (c + 1));
}

// Sum over the CSR entries q0..q1-1 of val[idx[q]], in ascending q, from 0 (the order of a
// plain loop, so the same bits), with the first 8 index loads and then the first 8 value
// loads issued together: the copies of a DOF cost two dependent memory latencies, not two
// per copy. TS: the type of the sum (the values are converted to it).
template <typename TS, typename TV>
__device__ __forceinline__ TS csr_sum(const int* __restrict__ idx, const TV* __restrict__ val, int q0, int q1) {
  constexpr int U = 8;
  int ix[U];
#pragma unroll
  for (int c = 0; c < U; ++c) ix[c] = (q0 + c < q1) ? idx[q0 + c] : 0;
  TV v[U];
#pragma unroll
  for (int c = 0; c < U; ++c)
    if (q0 + c < q1) v[c] = val[ix[c]];
  TS s = 0;
#pragma unroll
  for (int c = 0; c < U; ++c)
    if (q0 + c < q1) s += (TS)v[c];
  for (int q = q0 + U; q < q1; ++q) s += (TS)val[idx[q]];
  return s;
}

// Sum of the local copies of DOF g in wl (Eq. gather): one copy at a computed index for an
// interior DOF, the g2l CSR in ascending local order otherwise.
template <typename T>
__device__ __forceinline__ T gather_dof(const DevProblem& d, const T* __restrict__ wl, int g) {
  if (g < d.Gi) return wl[interior_local(d, g)];
  T s = 0;
  for (int q = d.g2l_off[g]; q < d.g2l_off[g + 1]; ++q) s += wl[d.g2l_idx[q]];
  return s;
}

// The same sum with the copies' loads issued together (csr_sum): faster in the gather pass
// of y = A x, where almost every DOF has several copies; the same bits.
template <typename T>
__device__ __forceinline__ T gather_dof_ilp(const DevProblem& d, const T* __restrict__ wl, int g) {
  if (g < d.Gi) return wl[interior_local(d, g)];
  return csr_sum<T, T>(d.g2l_idx, wl, d.g2l_off[g], d.g2l_off[g + 1]);
}


}  // namespace
}  // namespace sem
