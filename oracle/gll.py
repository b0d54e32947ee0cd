"""GLL nodes and weights, Lagrange basis and the derivative matrix.

Paper: Sec. 2.1 (Interpolation; Eq. D) and Sec. 2.4 (Integration).
Reading: the paper defines D_ij = phi_i'(t_j) (Eq. D) but uses sum_m D_im u_m for
d u/d xi at node i, which needs phi_m'(t_i). The oracle therefore builds
Dhat[i, m] = phi_m'(t_i) for gradients and uses its transpose for the
divergence (Algorithm 2 writes D_mi there).
Pinned by: closed-form nodes/weights for n = 1..4, exactness of the quadrature
for degree <= 2n-1 (and failure at 2n), nodes = roots of the library Legendre
derivative, Dhat = derivative of the product-formula basis, exactness of Dhat on
t^k for k <= n.
"""
import numpy as np


def legendre_and_derivative(n, t):
    """P_n(t) and P_n'(t) by the three-term recurrence and P_k' = t P_{k-1}' + k P_{k-1}."""
    t = np.asarray(t, dtype=np.float64)
    p_prev = np.ones_like(t)
    dp_prev = np.zeros_like(t)
    if n == 0:
        return p_prev, dp_prev
    p = t.copy()
    dp = np.ones_like(t)
    for k in range(2, n + 1):
        p_next = ((2 * k - 1) * t * p - (k - 1) * p_prev) / k
        dp_next = t * dp + k * p
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
    return p, dp


def gll_nodes_weights(n):
    """GLL points t_0 < ... < t_n on [-1, 1] and weights rho_i = 2 / (n(n+1) P_n(t_i)^2).

    Interior points are the roots of P_n', found by Newton's method; P_n'' comes
    from Legendre's equation (1 - t^2) P'' = 2 t P' - n(n+1) P.
    """
    if n < 1:
        raise ValueError("order must be >= 1")
    t = -np.cos(np.pi * np.arange(n + 1) / n)        # Chebyshev-Lobatto start
    for _ in range(100):
        p, dp = legendre_and_derivative(n, t[1:-1])
        ddp = (2 * t[1:-1] * dp - n * (n + 1) * p) / (1 - t[1:-1] ** 2)
        step = dp / ddp
        t[1:-1] -= step
        if np.all(np.abs(step) < 1e-16):
            break
    t[0], t[-1] = -1.0, 1.0
    p, _ = legendre_and_derivative(n, t)
    rho = 2.0 / (n * (n + 1) * p ** 2)
    return t, rho


def lagrange_basis(tn, x):
    """phi_j(x) for the Lagrange interpolants on nodes tn: returns array [len(x), len(tn)]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(tn)
    out = np.ones((len(x), m))
    for j in range(m):
        for l in range(m):
            if l != j:
                out[:, j] *= (x - tn[l]) / (tn[j] - tn[l])
    return out


def lagrange_basis_derivative(tn, x):
    """phi_j'(x) by differentiating the product formula term by term: [len(x), len(tn)]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(tn)
    out = np.zeros((len(x), m))
    for j in range(m):
        for l in range(m):
            if l == j:
                continue
            term = np.full(len(x), 1.0 / (tn[j] - tn[l]))
            for q in range(m):
                if q != j and q != l:
                    term *= (x - tn[q]) / (tn[j] - tn[q])
            out[:, j] += term
    return out


def derivative_matrix(n):
    """Dhat[i, m] = phi_m'(t_i) from the closed form for GLL nodes:
    P_n(t_i) / (P_n(t_m) (t_i - t_m)) for i != m, -n(n+1)/4 at (0,0), +n(n+1)/4 at (n,n), else 0."""
    t, _ = gll_nodes_weights(n)
    p, _ = legendre_and_derivative(n, t)
    D = np.zeros((n + 1, n + 1))
    for i in range(n + 1):
        for m in range(n + 1):
            if i != m:
                D[i, m] = p[i] / (p[m] * (t[i] - t[m]))
    D[0, 0] = -n * (n + 1) / 4.0
    D[n, n] = n * (n + 1) / 4.0
    return D
