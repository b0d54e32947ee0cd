// Test-only C entry points around the double-FP32 arithmetic of the FP64 element kernels
// (paper_1506_05996_gb300/csrc/kdw.cuh), compiled for the host, so that its error-free
// transforms and conversions can be checked against exact rational arithmetic on the CPU.
#include <cstdint>

#include "../paper_1506_05996_gb300/csrc/kdw.cuh"
#include "../paper_1506_05996_gb300/csrc/kgeomdw.cuh"

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

// The recomputed metric of the pair operator at the p^3 nodes of one element, staged as the
// element kernel stages it: the 8 binary64 vertices xyz[corner*3 + dim] taken relative to
// corner 0 in binary64 and split to pairs (absolute = 1: the coordinates split as they are,
// for the test that shows why the kernel does not); phi[2i] = (1 - t_i)/2, phi[2i + 1] = (1 + t_i)/2
// and w3[i + p (j + p k)] = rho_i rho_j rho_k split to nearest (the set-up tables). Results
// joined to binary64: G[c p^3 + node] for c < 6, m[node].
void dwh_geom(const double* xyz, const double* phi, const double* w3, int p, int absolute, double* G, double* m) {
  sem::dw xv[24], ph[2 * 16];
  for (int q = 0; q < 24; ++q) xv[q] = sem::dw_split(absolute ? xyz[q] : xyz[q] - xyz[q % 3]);
  for (int q = 0; q < 2 * p; ++q) ph[q] = sem::dw_split_host(phi[q]);
  const int p3 = p * p * p;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) {   // one line (i, j), k varying, as one thread of the kernel
      sem::LineJ L;
      sem::geom_line_dw(xv, ph + 2 * i, ph + 2 * j, L);
      for (int k = 0; k < p; ++k) {
        const int l = i + p * (j + p * k);
        sem::dw g[6], mm;
        sem::geom_node_dw(L, ph + 2 * k, sem::dw_split_host(w3[l]), g, mm);
        for (int c = 0; c < 6; ++c) G[c * p3 + l] = sem::dw_join(g[c]);
        m[l] = sem::dw_join(mm);
      }
    }
}

}
