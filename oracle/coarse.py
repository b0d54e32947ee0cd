"""Coarse-grid correction P^c r = m^{-1} C^T P_0 C m^{-1} r (Sec. 4.1, Eq. coarse).

Steps in the paper's order: y = r / m_N; scatter y; R_{IJK;e} = sum_ijk B_{IJK,ijk} y_{ijk;e}
m_{ijk;e}; gather R to the mesh vertices; Z = P_0 R; scatter Z; z_{ijk;e} =
sum_IJK B_{IJK,ijk} Z_{IJK;e} m_{ijk;e}; gather z; divide by m_N.
B_{IJK,ijk} = Phi_I(t_i) Phi_J(t_j) Phi_K(t_k) with Phi_0 = (1-t)/2, Phi_1 = (1+t)/2
(the paper prints its size as 8 x n^3; it is 8 x (n+1)^3).
Readings: the last step gathers (sums) z and scales z (not y) by 1/m_N; the coarse
space is the Q1 space on the free (non-Dirichlet) vertices; the coarse matrix A_0 is
the same operator at n = 1 (2-point GLL quadrature = the vertices), same lambda.
Pinned by: m^{-1} C^T reproduces the GLL-node coordinates from the vertex
coordinates (trilinear geometry), m^{-1} C^T 1 = 1, <C m^{-1} x, Y> = <x, m^{-1} C^T Y>,
A_0 equals the n = 1 assembled matrix, and with an exact P_0 the correction equals
Pi A_0^{-1} Pi^T computed densely.
"""
import numpy as np

from synth import VTK_CORNER_BITS


def vandermonde(t):
    """B[c, i, j, k] = Phi_{b0}(t_i) Phi_{b1}(t_j) Phi_{b2}(t_k) for VTK corner c with bits b."""
    Phi = np.stack([(1 - t) / 2, (1 + t) / 2])          # [bit, node]
    p = len(t)
    B = np.zeros((8, p, p, p))
    for c, (a, b, d) in enumerate(VTK_CORNER_BITS):
        B[c] = Phi[a][:, None, None] * Phi[b][None, :, None] * Phi[d][None, None, :]
    return B


def restrict(r, l2g, m_loc, m_N, B, hex2vert, n_vert):
    """Vertex vector R = C m^{-1} r (all vertices)."""
    y = r / m_N
    yl = y[l2g]
    Re = np.einsum("cijk,eijk->ec", B, yl * m_loc)
    return np.bincount(hex2vert.ravel(), weights=Re.ravel(), minlength=n_vert)


def prolong(Z, l2g, m_loc, m_N, B, hex2vert):
    """Global vector m^{-1} C^T Z from vertex values Z."""
    Ze = Z[hex2vert]                                     # [e, c]
    zl = np.einsum("cijk,ec->eijk", B, Ze) * m_loc
    z = np.bincount(l2g.ravel(), weights=zl.ravel(), minlength=m_N.shape[0])
    return z / m_N


def coarse_l2g(hex2vert):
    """Local-to-global table of the n = 1 space: node (i, j, k) in {0,1}^3 is a vertex."""
    lut = np.zeros((2, 2, 2), dtype=np.int64)
    for c, (a, b, d) in enumerate(VTK_CORNER_BITS):
        lut[a, b, d] = c
    E = hex2vert.shape[0]
    out = np.zeros((E, 2, 2, 2), dtype=np.int64)
    for a in range(2):
        for b in range(2):
            for d in range(2):
                out[:, a, b, d] = hex2vert[:, lut[a, b, d]]
    return out
