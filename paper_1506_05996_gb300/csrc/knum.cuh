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
#include "kgeomdw.cuh"

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

// Storage type of a kernel's local results: the pair's are joined to binary64.
template <typename T> struct LocalOf { using type = T; };
template <> struct LocalOf<dw> { using type = double; };

}  // namespace
}  // namespace sem
