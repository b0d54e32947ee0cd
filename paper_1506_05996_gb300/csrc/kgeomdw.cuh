// The recomputed metric of the double-FP32 operator (Sec. 2.3 geometry, Algorithm 2's
// pointwise factors), host and device: the element kernel calls it per line and per node, and
// the host build is checked against the binary64 factors on the CPU.
//
// G = w |J| J^-1 J^-T and m = w |J| at reference point (a, b, c), from the trilinear map of the
// 8 vertices xv[corner*3 + dim] (relative to any common origin: J does not depend on it). The
// reference-coordinate factors come as pairs, fa[0] = (1 - a)/2 and fa[1] = (1 + a)/2 (corner
// bit 0 / 1), and the same for b and c (a set-up table, split to nearest from binary64).
//
// The map is trilinear, so along a line of nodes with a and b fixed and c varying, the first
// two columns of J are fc[0] U + fc[1] V for per-line U and V, and the third column is
// constant. geom_line_dw forms U, V and that column once per line (the 72 corner
// multiply-accumulates); geom_node_dw completes J at a node with 6 products and 6
// multiply-accumulates, then takes the cofactors, the determinant and the scaled metric.
//
// The corner sums cancel (they add up to |J| from larger parts), which leaves the pairs' tails
// larger than half an ulp of their heads; a pair product drops tail x tail, so the sums are
// renormalised (one TwoSum each) before they are multiplied, and so are J's entries and the
// cofactors. On the 32^3 lattice the metric's worst error is about 17 u^2 (127 u^2 without
// the renormalisation).
#pragma once

#include "kdw.cuh"

namespace sem {

// The per-line part of J: J[r][0] = fc[0] U0[r][0] + fc[1] U0[r][1], the same with U1 for
// J[r][1], and J[r][2] = J2[r].
struct LineJ {
  dw U0[3][2];
  dw U1[3][2];
  dw J2[3];
};

DW_HD void geom_line_dw(const dw* xv, const dw* fa, const dw* fb, LineJ& L) {
  auto half = [](dw v) { return dw{0.5f * v.h, 0.5f * v.l}; };
  // d/da of corner q's basis function is +- fb[ib] fc[ic] / 2, d/db is +- fa[ia] fc[ic] / 2,
  // d/dc is +- fa[ia] fb[ib] / 2: the fc factor is left for the node
  const dw hb[2] = {half(fb[0]), half(fb[1])};
  const dw ha[2] = {half(fa[0]), half(fa[1])};
  dw ab[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) ab[u][v] = half(dw_mul(fa[u], fb[v]));
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    L.U0[r][0] = L.U0[r][1] = L.U1[r][0] = L.U1[r][1] = L.J2[r] = dw_zero();
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ia = ((q == 1) | (q == 2) | (q == 5) | (q == 6)) ? 1 : 0;   // VTK corner bits
    const int ib = ((q == 2) | (q == 3) | (q == 6) | (q == 7)) ? 1 : 0;
    const int ic = (q >= 4) ? 1 : 0;
    const dw d0 = ia ? hb[ib] : dw_neg(hb[ib]);
    const dw d1 = ib ? ha[ia] : dw_neg(ha[ia]);
    const dw d2 = ic ? ab[ia][ib] : dw_neg(ab[ia][ib]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const dw x = xv[3 * q + r];
      dw_mac(L.U0[r][ic], x, d0);
      dw_mac(L.U1[r][ic], x, d1);
      dw_mac(L.J2[r], x, d2);
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      L.U0[r][c] = dw_norm(L.U0[r][c]);
      L.U1[r][c] = dw_norm(L.U1[r][c]);
    }
    L.J2[r] = dw_norm(L.J2[r]);
  }
}

// G and m at the node of the line whose c factors are fc; w = rho_i rho_j rho_k as a pair.
DW_HD void geom_node_dw(const LineJ& L, const dw* fc, dw w, dw G[6], dw& m) {
  dw J[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    J[r][0] = dw_mul(fc[0], L.U0[r][0]);
    dw_mac(J[r][0], fc[1], L.U0[r][1]);
    J[r][1] = dw_mul(fc[0], L.U1[r][0]);
    dw_mac(J[r][1], fc[1], L.U1[r][1]);
    J[r][0] = dw_norm(J[r][0]);
    J[r][1] = dw_norm(J[r][1]);
    J[r][2] = L.J2[r];
  }
  auto cof = [](dw p, dw q, dw s, dw t) {   // p q - s t, renormalised
    dw v = dw_mul(p, q);
    dw_mac(v, dw_neg(s), t);
    return dw_norm(v);
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

}  // namespace sem
