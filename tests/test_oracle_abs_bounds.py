"""Pins for the two reference magnitudes of the reduced-precision bounds:
oracle.operator.matfree_abs (every term of Eq. R in absolute value) and
oracle.schwarz.apply_fine_abs (every term of Eq. z in absolute value).

Each is compared with a brute-force sum written term by term: for the operator, the
divergence index m, the metric entry (a, b) and the gradient index q of every product
D[m, i_a] G_ab D[node_b, q] u of Algorithm 2 / Eq. ABC; for the patch solve, every
(a, b, c) mode and every input box node of 8/(hx hy hz) S S S d^-1 S S S r. A dropped term,
a missing absolute value or a transposed D would change these sums. Both must also bound
the signed results they stand for: |A x| <= matfree_abs(x), |P^f r| <= apply_fine_abs(r).
"""
import itertools

import numpy as np
import pytest

from synth import lattice_hex_mesh
from oracle.problem import Problem
from oracle.operator import matfree_abs
from oracle.schwarz import apply_fine_abs

GIDX = ((0, 1, 2), (1, 3, 4), (2, 4, 5))   # G_ab -> stored entry (xx xy xz yy yz zz)


def brute_operator_abs(pr, x):
    """sum over every term of Eq. R in absolute value, gathered; masked rows 0."""
    p = pr.n + 1
    aD = np.abs(pr.Dh)                          # Dh[i, m] = phi_m'(t_i)
    u = np.where(pr.mask > 0, 0.0, np.abs(x))[pr.l2g]
    aG = np.abs(pr.Gf)
    out = np.zeros(pr.G)
    for e in range(pr.l2g.shape[0]):
        for i, j, k in itertools.product(range(p), repeat=3):
            out_ijk = (i, j, k)
            tot = pr.lam * pr.m_loc[e, i, j, k] * u[e, i, j, k]
            for a in range(3):                  # divergence direction
                for m in range(p):
                    node = list(out_ijk)
                    node[a] = m
                    cdiv = aD[m, out_ijk[a]]
                    for b in range(3):          # gradient direction
                        g = aG[GIDX[a][b], e, node[0], node[1], node[2]]
                        for q in range(p):
                            src = list(node)
                            src[b] = q
                            tot += cdiv * g * aD[node[b], q] * u[e, src[0], src[1], src[2]]
            out[pr.l2g[e, i, j, k]] += tot
    return np.where(pr.mask > 0, 0.0, out)


def brute_fine_abs(pr, r):
    """sum over every term of Eq. z (fast diagonalisation) in absolute value, per box,
    added into the global nodes of the box; masked rows 0."""
    P = pr.n + 3
    aS = np.abs(pr.S)
    ra = np.where(pr.mask > 0, 0.0, np.abs(r))
    out = np.zeros(pr.G)
    ev = pr.ev
    for e in range(pr.ip.shape[0]):
        hx, hy, hz = pr.h[e]
        ip = pr.ip[e]
        rb = np.where(ip >= 0, ra[np.where(ip >= 0, ip, 0)], 0.0)
        scale = 8.0 / (hx * hy * hz)
        # inverse eigenvalue sums d[a, b, c] > 0
        d = np.empty((P, P, P))
        for a, b, c in itertools.product(range(P), repeat=3):
            d[a, b, c] = 4.0 * (ev[a] / hx ** 2 + ev[b] / hy ** 2 + ev[c] / hz ** 2) + pr.lam
        # the modal amplitudes of |r| through |S|, one input node at a time
        t = np.zeros((P, P, P))
        for I2, J2, K2 in itertools.product(range(P), repeat=3):
            if rb[I2, J2, K2] != 0.0:
                t += rb[I2, J2, K2] * aS[I2][:, None, None] * aS[J2][None, :, None] * aS[K2][None, None, :]
        w = t / d
        for I, J, K in itertools.product(range(P), repeat=3):
            g = ip[I, J, K]
            if g < 0:
                continue
            out[g] += scale * np.sum(w * aS[I][:, None, None] * aS[J][None, :, None] * aS[K][None, None, :])
    return np.where(pr.mask > 0, 0.0, out)


@pytest.mark.parametrize("E,n,lam,a,seed,dirichlet", [(1, 3, 0.0, 0.2, 1, False), (2, 2, 1.7, 0.2, 2, True),
                                                      (2, 3, 0.6, 0.15, 3, False)])
def test_matfree_abs_is_the_sum_of_term_magnitudes(E, n, lam, a, seed, dirichlet):
    pr = Problem(lattice_hex_mesh(E, a, seed), n, lam, dirichlet=dirichlet, coarse_solver=None,
                 with_schwarz=False)
    x = np.random.default_rng(seed).standard_normal(pr.G)
    got = matfree_abs(x, pr.l2g, pr.Dh, pr.Gf, pr.m_loc, pr.lam, pr.mask)
    ref = brute_operator_abs(pr, x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(ref)
    # it bounds the signed apply on the free rows
    y = pr.apply_A(x)
    free = pr.mask == 0
    assert np.all(np.abs(y[free]) <= got[free] * (1 + 1e-12))
    # a sign-definite input with a nonnegative operator would give equality; here the
    # bound is not tight for random x
    assert np.max(np.abs(y[free]) / got[free]) < 1.0


@pytest.mark.parametrize("E,n,lam,a,seed", [(2, 2, 0.0, 0.2, 4), (2, 3, 1.3, 0.1, 5)])
def test_apply_fine_abs_is_the_sum_of_term_magnitudes(E, n, lam, a, seed):
    pr = Problem(lattice_hex_mesh(E, a, seed), n, lam, coarse_solver=None)
    r = np.random.default_rng(seed).standard_normal(pr.G)
    got = apply_fine_abs(r, pr.ip, pr.S, pr.ev, pr.h, pr.lam, pr.mask)
    ref = brute_fine_abs(pr, r)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(ref)
    z = pr.apply_Pf(r)
    free = pr.mask == 0
    assert np.all(np.abs(z[free]) <= got[free] * (1 + 1e-12))
    assert np.max(np.abs(z[free]) / got[free]) < 1.0
