// Double-FP32 ("double-word") arithmetic of the FP64 interface's element kernels.
//
// On GB300 the FP64 pipe issues about 2 multiply-adds per clock per SM, 1/64 of the FP32
// pipe, and the FP64 operator and patch-solve kernels saturate it. Their contractions run
// here instead on the FP32 pipe, on unevaluated pairs x = h + l of binary32 numbers
// (Dekker 1971; the error-free transforms TwoSum of Knuth and TwoProduct by FMA). Errors
// follow the usual sum-of-products model with the unit u^2 = 2^-48 instead of binary64's
// 2^-53: every step errs by a small multiple of 2^-48 times the magnitudes of its operands,
// so a p-term contraction errs by about p 2^-48 sum |a_i||b_i| (binary64: p 2^-53 of it).
//
// Operations (u = 2^-24):
//  dw_split   binary64 -> pair: h = x truncated to 24 significant bits, l = the next 23 bits
//             truncated, by integer operations on the IEEE-754 layout (the conversion
//             instruction runs on the FP64 pipe); |x - (h + l)| < 2^-46 |x| for
//             2^-80 <= |x| < 2^128; below 2^-80 l is 0 (relative error 2^-23), below
//             2^-126 the pair is a signed zero; infinities and NaNs carry over to h.
//  dw_join    pair -> binary64, by TwoSum and integer operations: the pair value rounded
//             toward zero to 53 bits (relative error below 2^-52 after the TwoSum).
//  dw_add     sloppy sum, not renormalised: (s, e) = TwoSum(x.h, y.h), l = e + (x.l + y.l);
//             error at most about 2u^2 (|x| + |y|).
//  dw_mac     acc += x y: TwoProduct of the high parts, the two cross products by FMA,
//             TwoSum into the accumulator's high part, every low-order term into its low
//             part; error at most about 3u^2 |x||y| per step plus the accumulated 2u^2 |acc|.
// The pairs a kernel keeps (shared-memory lines, accumulators) are not renormalised after
// every step: a low part that grew beyond ulp(h) still carries its exact share of the value
// and enters the next products through the cross terms, whose own rounding is then
// u |x.h| |l| = O(u^2) of the operands. That holds while one operand of each product is
// normalised (a table split at set-up, an input split from binary64): a product drops
// x.l y.l, and after a sum that cancels by a factor R both tails can reach u R of their heads,
// which makes the dropped term (u R)^2. Products of two computed pairs (the recomputed
// metric's J and cofactors) renormalise them first with dw_norm; dw_join renormalises too.
//
// Products are formed with the _rn intrinsics, which the compiler never contracts into an
// FMA (a contracted h = a b + c would break the error-free transforms).
#pragma once

#include <cstdint>
#include <cstring>
#include <cmath>

#ifdef __CUDACC__
#define DW_HD __host__ __device__ __forceinline__
#else
#define DW_HD inline
#endif

namespace sem {

struct dw {
  float h, l;   // the value h + l
};

DW_HD uint32_t dw_f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
DW_HD float dw_u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
DW_HD uint64_t dw_d2u(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}
DW_HD double dw_u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}

// Correctly rounded binary32 operations that are never fused.
DW_HD float dw_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
DW_HD float dw_sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float r = a - b;
  return r;
#endif
}
DW_HD float dw_mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
DW_HD float dw_fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// TwoSum (Knuth): s + e = a + b exactly, s = fl(a + b).
DW_HD dw dw_two_sum(float a, float b) {
  const float s = dw_add_rn(a, b);
  const float bb = dw_sub_rn(s, a);
  const float e = dw_add_rn(dw_sub_rn(a, dw_sub_rn(s, bb)), dw_sub_rn(b, bb));
  return {s, e};
}

DW_HD dw dw_zero() { return {0.0f, 0.0f}; }

DW_HD dw dw_add(dw x, dw y) {
  const dw s = dw_two_sum(x.h, y.h);
  return {s.h, dw_add_rn(s.l, dw_add_rn(x.l, y.l))};
}
DW_HD dw dw_sub(dw x, dw y) {
  const dw s = dw_two_sum(x.h, -y.h);
  return {s.h, dw_add_rn(s.l, dw_sub_rn(x.l, y.l))};
}
DW_HD dw dw_neg(dw x) { return {-x.h, -x.l}; }

// x y: TwoProduct of the high parts plus both cross products.
DW_HD dw dw_mul(dw x, dw y) {
  const float p = dw_mul_rn(x.h, y.h);
  float e = dw_fma_rn(x.h, y.h, -p);
  e = dw_fma_rn(x.h, y.l, e);
  e = dw_fma_rn(x.l, y.h, e);
  return {p, e};
}

// acc += x y
DW_HD void dw_mac(dw& acc, dw x, dw y) {
  const float p = dw_mul_rn(x.h, y.h);
  float e = dw_fma_rn(x.h, y.h, -p);
  e = dw_fma_rn(x.h, y.l, e);
  e = dw_fma_rn(x.l, y.h, e);
  const dw s = dw_two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = dw_add_rn(acc.l, dw_add_rn(s.l, e));
}

// Renormalised pair: |l| <= ulp(h) / 2.
DW_HD dw dw_norm(dw x) { return dw_two_sum(x.h, x.l); }

// x / y (double-word division, after Joldes, Muller and Popescu 2017, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", DWDivDW): the quotient's
// high part from the binary32 reciprocal of y.h, the exact remainder x - q_h y in pairs, and
// the low part from the remainder; relative error a few u^2 for normalised y.
DW_HD float dw_rcp_rn(float a) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(a);
#else
  volatile float r = 1.0f / a;
  return r;
#endif
}
DW_HD dw dw_div(dw x, dw y) {
  const dw yn = dw_norm(y);
  const float r = dw_rcp_rn(yn.h);
  const float qh = dw_mul_rn(x.h, r);
  // q_h y = TwoProduct(q_h, y.h) + q_h y.l
  const float p = dw_mul_rn(qh, yn.h);
  const float pe = dw_fma_rn(qh, yn.l, dw_fma_rn(qh, yn.h, -p));
  const dw rem = dw_sub(x, {p, pe});
  const float ql = dw_mul_rn(dw_add_rn(rem.h, rem.l), r);
  return dw_two_sum(qh, ql);
}

// binary64 -> pair (see the header comment).
DW_HD dw dw_split(double x) {
  const uint64_t b = dw_d2u(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);   // biased binary64 exponent
  const int eh = e - 896;                     // biased binary32 exponent of h (1023 - 127)
  // h: the top 23 fraction bits (20 of the high word, 3 of the low word)
  const float h = dw_u2f(sign | ((uint32_t)eh << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // l: fraction bits 28..6 as an integer k < 2^23, times 2^(e - 1023 - 46); k becomes a
  // binary32 exactly through the 2^23 magic constant
  const uint32_t k = (lw >> 6) & 0x7fffffu;
  const float kf = dw_sub_rn(dw_u2f(0x4b000000u | k), 8388608.0f);
  const int el = e - 942;                     // biased binary32 exponent of 2^(e - 1023 - 46)
  const float sc = dw_u2f(sign | ((uint32_t)(el > 0 ? el : 0) << 23));
  dw r = {h, el > 0 ? dw_mul_rn(kf, sc) : 0.0f};
  if (eh <= 0) r = {dw_u2f(sign), 0.0f};     // zero, subnormal, or below binary32's range
  if (eh >= 255) {                            // beyond binary32's range, infinity or NaN
    const bool nan = e == 0x7ff && (((hw & 0xfffffu) | lw) != 0u);
    r = {dw_u2f(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.0f};
  }
  return r;
}

// pair -> binary64 (see the header comment).
DW_HD double dw_join(dw x) {
  const dw n = dw_two_sum(x.h, x.l);   // |n.l| <= ulp(n.h) / 2
  const uint32_t hb = dw_f2u(n.h), lb = dw_f2u(n.l);
  const int eh = (int)((hb >> 23) & 0xffu), el = (int)((lb >> 23) & 0xffu);
  const uint64_t sh = (uint64_t)(hb & 0x80000000u) << 32;
  if (eh == 0xff) return dw_u2d(sh | 0x7ff0000000000000ull | ((uint64_t)(hb & 0x7fffffu) << 29));
  if (eh == 0) return dw_u2d(sh);       // zero (binary32 subnormal high parts are dropped)
  // significand of h as 53 bits: (2^23 + fraction) 2^29, in units of 2^(eh - 127 - 52)
  uint64_t M = ((uint64_t)((hb & 0x7fffffu) | 0x800000u)) << 29;
  if (el != 0) {
    // l = (2^23 + fraction) 2^(el - 127 - 23) = (2^23 + fraction) 2^(el - eh + 29) units;
    // el <= eh - 24, so the shift is at most 5 to the left
    const uint64_t ml = (uint64_t)((lb & 0x7fffffu) | 0x800000u);
    const int s = el - eh + 29;
    const uint64_t c = s >= 0 ? (ml << s) : (s > -40 ? (ml >> (-s)) : 0ull);
    M = ((hb ^ lb) & 0x80000000u) ? M - c : M + c;
  }
  int ex = eh - 127 + 1023;
  if (M < (1ull << 52)) {               // h a power of two and l of the other sign
    M <<= 1;
    ex -= 1;
  }
  return dw_u2d(sh | ((uint64_t)ex << 52) | (M & 0xfffffffffffffull));
}

// A host-side split of a table constant, to nearest: h = fl32(x), l = fl32(x - h).
inline dw dw_split_host(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

}  // namespace sem
