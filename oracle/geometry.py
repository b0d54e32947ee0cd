"""Element geometry at GLL nodes (Sec. 2.3 Geometry, Sec. 2.4 Integration).

Trilinear map x^e(xi, eta, zeta) = sum_v x_v N_v with N_v = prod (1 + s_v t)/2 over
the VTK corner signs s_v; J[a, b] = d x_a / d xi_b.
Readings: the paper calls the metric G = J^T J; the stiffness needs
G = rho_i rho_j rho_k |J| J^{-1} J^{-T} (the weight and |J| folded in, Algorithm 2
applies m only to the c-term). G1..G6 = (xx, xy, xz, yy, yz, zz) entries of that
symmetric matrix in reference coordinates, matching the row pattern of Eq. R / Eq. ABC.
m_{ijk;e} = rho_i rho_j rho_k |J|.
Pinned by: sum of m = volume of the mesh (unit cube), per-element sum of m = the
trilinear volume from 2x2x2 Gauss quadrature, affine meshes reproduce |a|^2 vol
for the energy of linear functions (operator tests).
"""
import numpy as np

from synth import VTK_CORNER_BITS


def jacobians(xyz_e, t):
    """J[e, i, j, k, a, b] = d x_a / d xi_b at GLL node (t_i, t_j, t_k)."""
    s = (2 * VTK_CORNER_BITS - 1).astype(np.float64)
    p = len(t)
    J = np.zeros((xyz_e.shape[0], p, p, p, 3, 3))
    for c in range(8):
        fx = (1 + s[c, 0] * t) / 2
        fy = (1 + s[c, 1] * t) / 2
        fz = (1 + s[c, 2] * t) / 2
        dN = np.zeros((p, p, p, 3))
        dN[..., 0] = (s[c, 0] / 2) * fy[None, :, None] * fz[None, None, :] * np.ones((p, 1, 1))
        dN[..., 1] = fx[:, None, None] * (s[c, 1] / 2) * fz[None, None, :] * np.ones((1, p, 1))
        dN[..., 2] = fx[:, None, None] * fy[None, :, None] * (s[c, 2] / 2) * np.ones((1, 1, p))
        J += xyz_e[:, c, None, None, None, :, None] * dN[None, :, :, :, None, :]
    return J


def geometric_factors(xyz_e, t, rho):
    """Return (G [6, E, p, p, p], m [E, p, p, p], detJ [E, p, p, p])."""
    J = jacobians(xyz_e, t)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    w = rho[:, None, None] * rho[None, :, None] * rho[None, None, :]
    Gm = np.einsum("...ac,...bc->...ab", Jinv, Jinv) * (w[None] * detJ)[..., None, None]
    G = np.stack([Gm[..., 0, 0], Gm[..., 0, 1], Gm[..., 0, 2],
                  Gm[..., 1, 1], Gm[..., 1, 2], Gm[..., 2, 2]])
    m = w[None] * detJ
    return G, m, detJ


def element_box_sizes(xyz_e):
    """h_x, h_y, h_z per element: mean length of the 4 element edges along xi, eta, zeta.

    Reading of Sec. 4.2 ("each hexahedron is approximated as a parallelogram of
    dimensions h_x, h_y, h_z"), which does not say how h is measured.
    """
    out = np.zeros((xyz_e.shape[0], 3))
    for ax in range(3):
        lens = []
        for c in range(8):
            if VTK_CORNER_BITS[c, ax] == 0:
                bits = VTK_CORNER_BITS[c].copy()
                bits[ax] = 1
                c2 = int(np.where((VTK_CORNER_BITS == bits).all(axis=1))[0][0])
                lens.append(np.linalg.norm(xyz_e[:, c2] - xyz_e[:, c], axis=1))
        out[:, ax] = np.mean(lens, axis=0)
    return out
