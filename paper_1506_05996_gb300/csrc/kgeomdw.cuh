// The recomputed metric of the double-FP32 operator (Sec. 2.3 geometry, Algorithm 2's
// pointwise factors), host and device: the element kernel calls it per node, and the host
// build is checked against the binary64 factors on the CPU.
#pragma once

#include "kdw.cuh"

namespace sem {

// G = w |J| J^-1 J^-T and m = w |J| at reference point (a, b, c) in pair arithmetic (the
// recomputed-geometry form of the double-FP32 operator): the trilinear map's Jacobian from the
// 8 vertices xv[corner*3 + dim] (relative to any common origin: J does not depend on it), its
// cofactors, determinant and the scaled metric, the same steps as geom_point in kcommon.cuh.
// The reference-coordinate factors come as pairs: fa[0] = (1 - a)/2, fa[1] = (1 + a)/2 (corner
// bit 0 / 1), and the same for b and c (a set-up table, split to nearest from binary64).
DW_HD void geom_point_dw(const dw* xv, const dw* fa, const dw* fb, const dw* fc, dw w, dw G[6], dw& m) {
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
  // The sums above cancel (the corner terms add up to |J| from larger parts), which leaves the
  // pairs' tails larger than half an ulp of their heads; a pair product drops tail x tail, so
  // J, and below the cofactors, are renormalised before they are multiplied (one TwoSum per
  // entry; on the 32^3 lattice the metric's worst error falls from 127 to 20 u^2).
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) J[r][s] = dw_norm(J[r][s]);
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
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) C[r][s] = dw_norm(C[r][s]);
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
