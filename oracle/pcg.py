"""Preconditioned conjugate gradients (Algorithm 1).

Readings: r = b - A u, so with u_0 = 0 the first residual is b, and f = A p_k;
the stopping test, which the paper does not state, is ||r_k||_2 <= rtol ||b||_2
on the recursively updated residual, checked after each residual update; the
returned iteration count is the number of operator applications.
Pinned by: with P = I on a dense SPD matrix the iterates are the CG iterates
(A-orthogonal directions, residual recurrence equals b - A u), and the converged
solution equals a direct solve.

fpcg: the flexible variant for a preconditioner that changes between applications (the
K-cycle of Sec. 4.1): beta_k = z_k.(r_k - r_k-1) / (z_k-1.r_k-1) (Polak-Ribiere form), the
rest as Algorithm 1. Pinned by: with a fixed SPD preconditioner it takes the iterations of
pcg (z_k.r_k-1 = 0 then).
"""
import numpy as np


def pcg(apply_A, apply_P, b, rtol=1e-8, maxit=1000):
    u = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    if hist[0] <= rtol:
        return u, 0, np.array(hist)
    z = apply_P(r)
    p = z.copy()
    rz = z @ r
    it = 0
    while it < maxit:
        f = apply_A(p)
        alpha = rz / (p @ f)
        u = u + alpha * p
        r = r - alpha * f
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= rtol:
            break
        z = apply_P(r)
        rz_new = z @ r
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return u, it, np.array(hist)


def fpcg(apply_A, apply_P, b, rtol=1e-8, maxit=1000):
    u = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    if hist[0] <= rtol:
        return u, 0, np.array(hist)
    z = apply_P(r)
    p = z.copy()
    rz = z @ r
    it = 0
    while it < maxit:
        f = apply_A(p)
        alpha = rz / (p @ f)
        u = u + alpha * p
        r_prev = r
        r = r - alpha * f
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= rtol:
            break
        z = apply_P(r)
        rz_new = z @ r
        beta = (rz_new - z @ r_prev) / rz
        rz = rz_new
        p = z + beta * p
    return u, it, np.array(hist)
