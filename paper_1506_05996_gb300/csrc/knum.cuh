// Arithmetic of the element kernels, written once for their three number types:
// double (binary64 on the FP64 pipe), float (binary32, the mixed path) and dw (a pair of
// binary32 numbers, kdw.cuh: the FP64 interface's kernels on the FP32 pipe).
// For double and float every helper is the plain expression the kernels used before
// (a += x * y and friends, which the compiler contracts to the same fused multiply-adds),
// so those instantiations are unchanged.
#pragma once

#include <cuda_bf16.h>
#include <type_traits>

#include "device.h"
#include "kdw.cuh"

namespace sem {
namespace {

template <typename T> constexpr bool kIsDw = std::is_same<T, dw>::value;

template <typename T> __device__ __forceinline__ T num_zero() { return T(0); }
template <> __device__ __forceinline__ dw num_zero<dw>() { return dw_zero(); }

__device__ __forceinline__ float num_add(float a, float b) { return a + b; }
__device__ __forceinline__ double num_add(double a, double b) { return a + b; }
__device__ __forceinline__ dw num_add(dw a, dw b) { return dw_add(a, b); }
__device__ __forceinline__ float num_sub(float a, float b) { return a - b; }
__device__ __forceinline__ double num_sub(double a, double b) { return a - b; }
__device__ __forceinline__ dw num_sub(dw a, dw b) { return dw_sub(a, b); }
__device__ __forceinline__ float num_mul(float a, float b) { return a * b; }
__device__ __forceinline__ double num_mul(double a, double b) { return a * b; }
__device__ __forceinline__ dw num_mul(dw a, dw b) { return dw_mul(a, b); }
// acc += x y
__device__ __forceinline__ void num_mac(float& acc, float x, float y) { acc += x * y; }
__device__ __forceinline__ void num_mac(double& acc, double x, double y) { acc += x * y; }
__device__ __forceinline__ void num_mac(dw& acc, dw x, dw y) { dw_mac(acc, x, y); }
// a b + c
__device__ __forceinline__ float num_fma(float a, float b, float c) { return a * b + c; }
__device__ __forceinline__ double num_fma(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ dw num_fma(dw a, dw b, dw c) {
  dw_mac(c, a, b);
  return c;
}
// a0 b0 + a1 b1 + a2 b2
template <typename T>
__device__ __forceinline__ T num_dot3(T a0, T b0, T a1, T b1, T a2, T b2) {
  if constexpr (kIsDw<T>) {
    dw s = dw_mul(a0, b0);
    dw_mac(s, a1, b1);
    dw_mac(s, a2, b2);
    return s;
  } else {
    return a0 * b0 + a1 * b1 + a2 * b2;
  }
}

// A global-vector entry (binary64 or binary32) as the kernel's number type: the pair
// by the integer split of kdw.cuh.
template <typename T> __device__ __forceinline__ T num_load(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T num_load(float v) { return (T)v; }
template <> __device__ __forceinline__ dw num_load<dw>(double v) { return dw_split(v); }

// A table constant (set-up data in binary64) as the kernel's number type: the pair to
// nearest (h = fl32(v), l = fl32(v - h)), read once per CTA.
template <typename T> __device__ __forceinline__ T num_const(double v) { return (T)v; }
template <> __device__ __forceinline__ dw num_const<dw>(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

// A kernel result stored into a global array of type TO.
template <typename TO> __device__ __forceinline__ TO num_store(double v) { return (TO)v; }
template <typename TO> __device__ __forceinline__ TO num_store(float v) { return (TO)v; }
template <typename TO> __device__ __forceinline__ TO num_store(dw v) { return (TO)dw_join(v); }
template <> __device__ __forceinline__ dw num_store<dw>(dw v) { return v; }   // pairs kept as pairs

// The stored factors as pairs (SEM_PREC_FP64 on the FP32 pipe).
template <typename T> __device__ __forceinline__ T factor(dw v) { return v; }
template <typename T> __device__ __forceinline__ const T* geo_of(const DevProblem& d);
template <> __device__ __forceinline__ const dw* geo_of<dw>(const DevProblem& d) { return d.geodw; }

// G = w |J| J^-1 J^-T and m = w |J| at reference point (a, b, c) in pair arithmetic (the
// recomputed-geometry form of the double-FP32 operator): the trilinear map's Jacobian from the
// 8 vertices xv[corner*3 + dim] (relative to any common origin: J does not depend on it), its
// cofactors, determinant and the scaled metric, the same steps as geom_point in kcommon.cuh.
// The reference-coordinate factors come as pairs: fa[0] = (1 - a)/2, fa[1] = (1 + a)/2 (corner
// bit 0 / 1), and the same for b and c (a set-up table, split to nearest from binary64).
__device__ __forceinline__ void geom_point_dw(const dw* xv, const dw* fa, const dw* fb, const dw* fc, dw w, dw G[6],
                                              dw& m) {
  auto half = [](dw v) { return dw{0.5f * v.h, 0.5f * v.l}; };
  // d/da of the corner's basis function is +- fb fc / 2, and so on
  dw bc[2][2], ac[2][2], ab[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      bc[u][v] = half(dw_mul(fb[u], fc[v]));
      ac[u][v] = half(dw_mul(fa[u], fc[v]));
      ab[u][v] = half(dw_mul(fa[u], fb[v]));
    }
  dw J[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) J[r][s] = dw_zero();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ia = ((q == 1) | (q == 2) | (q == 5) | (q == 6)) ? 1 : 0;   // VTK corner bits
    const int ib = ((q == 2) | (q == 3) | (q == 6) | (q == 7)) ? 1 : 0;
    const int ic = (q >= 4) ? 1 : 0;
    const dw d0 = ia ? bc[ib][ic] : dw_neg(bc[ib][ic]);
    const dw d1 = ib ? ac[ia][ic] : dw_neg(ac[ia][ic]);
    const dw d2 = ic ? ab[ia][ib] : dw_neg(ab[ia][ib]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const dw x = xv[3 * q + r];
      dw_mac(J[r][0], x, d0);
      dw_mac(J[r][1], x, d1);
      dw_mac(J[r][2], x, d2);
    }
  }
  auto cof = [](dw p, dw q, dw s, dw t) {   // p q - s t
    dw v = dw_mul(p, q);
    dw_mac(v, dw_neg(s), t);
    return v;
  };
  dw C[3][3];
  C[0][0] = cof(J[1][1], J[2][2], J[1][2], J[2][1]);
  C[0][1] = cof(J[1][2], J[2][0], J[1][0], J[2][2]);
  C[0][2] = cof(J[1][0], J[2][1], J[1][1], J[2][0]);
  C[1][0] = cof(J[0][2], J[2][1], J[0][1], J[2][2]);
  C[1][1] = cof(J[0][0], J[2][2], J[0][2], J[2][0]);
  C[1][2] = cof(J[0][1], J[2][0], J[0][0], J[2][1]);
  C[2][0] = cof(J[0][1], J[1][2], J[0][2], J[1][1]);
  C[2][1] = cof(J[0][2], J[1][0], J[0][0], J[1][2]);
  C[2][2] = cof(J[0][0], J[1][1], J[0][1], J[1][0]);
  dw det = dw_mul(J[0][0], C[0][0]);
  dw_mac(det, J[0][1], C[0][1]);
  dw_mac(det, J[0][2], C[0][2]);
  const dw sc = dw_div(w, det);   // inv(J)[r][c] = C[c][r] / det
  auto col = [&](int i, int j) {
    dw v = dw_mul(C[0][i], C[0][j]);
    dw_mac(v, C[1][i], C[1][j]);
    dw_mac(v, C[2][i], C[2][j]);
    return dw_mul(sc, v);
  };
  G[0] = col(0, 0);
  G[1] = col(0, 1);
  G[2] = col(0, 2);
  G[3] = col(1, 1);
  G[4] = col(1, 2);
  G[5] = col(2, 2);
  m = dw_mul(w, det);
}

// Storage type of a kernel's local results: the pair's are joined to binary64.
template <typename T> struct LocalOf { using type = T; };
template <> struct LocalOf<dw> { using type = double; };

}  // namespace
}  // namespace sem
