"""Screened-Poisson operator: matrix-free residual and explicit assembly.

Paper: weak form Eq. pdeweak; residual Eq. R; Algorithm 2 with Eq. ABC.
Readings: kappa = 1 and c = lam >= 0 constant; the quadrature weights live in G
(G = w |J| J^{-1} J^{-T}) and m multiplies only the c-term (Algorithm 2);
Dhat[i, m] = phi_m'(t_i) for the gradient and its transpose for the divergence.
Dirichlet conditions by masking: rows/columns of masked nodes are dropped and
replaced by the identity, A_D = P_f A P_f + P_d.

matfree_local follows Algorithm 2 step by step (gradient, A/B/C, transposed
contraction plus c m u). element_matrices builds each A_e basis function by
basis function from the product-formula Lagrange basis and J^{-T} (no sum
factorisation), so the two are independent computations of the same operator.
Pinned by: matrix-free == assembled on tiny meshes, symmetry, A 1 = lam m with no
mask, zero rows for linear functions at interior nodes of affine meshes, energy of a
linear function = |a|^2 vol on affine meshes, SPD under Dirichlet.
"""
import numpy as np
from scipy.sparse import coo_matrix

from .gll import lagrange_basis, lagrange_basis_derivative


def matfree_local(u, Dh, G, m, lam):
    """Local residual r_{ijk;e} from local values u[e, i, j, k] (Algorithm 2)."""
    ur = np.einsum("im,emjk->eijk", Dh, u)       # d u / d xi   at (i, j, k)
    us = np.einsum("jm,eimk->eijk", Dh, u)       # d u / d eta
    ut = np.einsum("km,eijm->eijk", Dh, u)       # d u / d zeta
    A = G[0] * ur + G[1] * us + G[2] * ut
    B = G[1] * ur + G[3] * us + G[4] * ut
    C = G[2] * ur + G[4] * us + G[5] * ut
    r = (np.einsum("mi,emjk->eijk", Dh, A)
         + np.einsum("mj,eimk->eijk", Dh, B)
         + np.einsum("mk,eijm->eijk", Dh, C))
    return r + lam * m * u


def matfree_apply(x, l2g, Dh, G, m, lam, mask=None):
    """y = A_D x: scatter, local residual, gather; masked rows return x."""
    Gn = int(x.shape[0])
    xf = x if mask is None else np.where(mask > 0, 0.0, x)
    r = matfree_local(xf[l2g], Dh, G, m, lam)
    y = np.bincount(l2g.ravel(), weights=r.ravel(), minlength=Gn)
    if mask is not None:
        y = np.where(mask > 0, x, y)
    return y


def element_matrices(t, rho, J, lam):
    """Dense A_e[a, b] = sum_q w_q |J_q| grad phi_a(q) . grad phi_b(q) + lam sum_q w_q |J_q| phi_a(q) phi_b(q).

    grad phi_a(q) = J^{-T}(q) (phi'_{a1} phi_{a2} phi_{a3}, phi_{a1} phi'_{a2} phi_{a3},
    phi_{a1} phi_{a2} phi'_{a3}) evaluated at the GLL node q, basis index a = (a1, a2, a3)
    flattened in C order over (i, j, k), the order of l2g[e].reshape(-1).
    """
    p = len(t)
    phi = lagrange_basis(t, t)          # [q, a] = phi_a(t_q)
    dphi = lagrange_basis_derivative(t, t)
    # reference gradients g[a1,a2,a3, q1,q2,q3, 3]
    g0 = np.einsum("xa,yb,zc->abcxyz", dphi, phi, phi)
    g1 = np.einsum("xa,yb,zc->abcxyz", phi, dphi, phi)
    g2 = np.einsum("xa,yb,zc->abcxyz", phi, phi, dphi)
    gref = np.stack([g0, g1, g2], axis=-1).reshape(p ** 3, p ** 3, 3)   # [a, q, 3]
    val = np.einsum("xa,yb,zc->abcxyz", phi, phi, phi).reshape(p ** 3, p ** 3)
    w = (rho[:, None, None] * rho[None, :, None] * rho[None, None, :]).reshape(p ** 3)
    Jq = J.reshape(J.shape[0], p ** 3, 3, 3)
    Jinv = np.linalg.inv(Jq)
    detJ = np.linalg.det(Jq)
    W = w[None, :] * detJ                                 # [e, q]
    grad = np.einsum("eqba,xqb->exqa", Jinv, gref)        # J^{-T} gref : [e, a, q, 3]
    Ae = np.einsum("exqd,eq,eyqd->exy", grad, W, grad)
    Ae += lam * np.einsum("xq,eq,yq->exy", val, W, val)
    return Ae


def assemble(Ae, l2g, G):
    """Sparse global matrix (CSR) from element matrices with the local-to-global table."""
    E = Ae.shape[0]
    idx = l2g.reshape(E, -1)
    rows = np.repeat(idx[:, :, None], idx.shape[1], axis=2)
    cols = np.repeat(idx[:, None, :], idx.shape[1], axis=1)
    return coo_matrix((Ae.ravel(), (rows.ravel(), cols.ravel())), shape=(G, G)).tocsr()


def apply_dirichlet(A, mask):
    """A_D = P_f A P_f + P_d for a 0/1 mask (1 = Dirichlet node)."""
    from scipy.sparse import diags
    f = (mask == 0).astype(np.float64)
    Pf = diags(f)
    return (Pf @ A @ Pf + diags(1.0 - f)).tocsr()


def matfree_abs(x, l2g, Dh, G, m, lam, mask=None):
    """Magnitude of every term of Eq. R: the matrix-free apply with |D|, |G|, |x| and
    every sum taken over absolute values, gathered. Rounding bounds of a
    reduced-precision apply are multiples of this vector (a standard bound for sums of
    products: |fl(sum a_i b_i) - sum a_i b_i| <= gamma_K sum |a_i||b_i|)."""
    Gn = int(x.shape[0])
    xf = np.abs(x) if mask is None else np.where(mask > 0, 0.0, np.abs(x))
    u = xf[l2g]
    aD = np.abs(Dh)
    aG = np.abs(G)
    ur = np.einsum("im,emjk->eijk", aD, u)
    us = np.einsum("jm,eimk->eijk", aD, u)
    ut = np.einsum("km,eijm->eijk", aD, u)
    A = aG[0] * ur + aG[1] * us + aG[2] * ut
    B = aG[1] * ur + aG[3] * us + aG[4] * ut
    C = aG[2] * ur + aG[4] * us + aG[5] * ut
    r = (np.einsum("mi,emjk->eijk", aD, A) + np.einsum("mj,eimk->eijk", aD, B)
         + np.einsum("mk,eijm->eijk", aD, C)) + lam * m * u
    y = np.bincount(l2g.ravel(), weights=r.ravel(), minlength=Gn)
    if mask is not None:
        y = np.where(mask > 0, 0.0, y)
    return y
