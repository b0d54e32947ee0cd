// Test-only C entry points around the double-FP32 arithmetic of the FP64 element kernels
// (paper_1506_05996_gb300/csrc/kdw.cuh), compiled for the host, so that its error-free
// transforms and conversions can be checked against exact rational arithmetic on the CPU.
#include <cstdint>

#include "../paper_1506_05996_gb300/csrc/kdw.cuh"

extern "C" {

void dwh_split(const double* x, float* h, float* l, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    const sem::dw d = sem::dw_split(x[i]);
    h[i] = d.h;
    l[i] = d.l;
  }
}

void dwh_join(const float* h, const float* l, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = sem::dw_join({h[i], l[i]});
}

// op 0: x + y, 1: x - y, 2: x * y, 3: acc + x * y (acc in ah, al), 4: x / y
void dwh_op(int op, const float* xh, const float* xl, const float* yh, const float* yl, float* ah, float* al,
            int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    const sem::dw x = {xh[i], xl[i]}, y = {yh[i], yl[i]};
    sem::dw r;
    if (op == 0) r = sem::dw_add(x, y);
    else if (op == 1) r = sem::dw_sub(x, y);
    else if (op == 2) r = sem::dw_mul(x, y);
    else if (op == 4) r = sem::dw_div(x, y);
    else {
      r = {ah[i], al[i]};
      sem::dw_mac(r, x, y);
    }
    ah[i] = r.h;
    al[i] = r.l;
  }
}

// sum_k a[i*k + j] b[i*k + j] over j < k with dw_mac from zero, for each i; the pairs are
// split from binary64 inputs, and the result joined back
void dwh_dot(const double* a, const double* b, double* out, int64_t n, int k) {
  for (int64_t i = 0; i < n; ++i) {
    sem::dw acc = sem::dw_zero();
    for (int j = 0; j < k; ++j) sem::dw_mac(acc, sem::dw_split(a[i * k + j]), sem::dw_split(b[i * k + j]));
    out[i] = sem::dw_join(acc);
  }
}

}
