"""The double-FP32 arithmetic of the FP64 element kernels (csrc/kdw.cuh), built for the
host and checked against exact rational arithmetic (fractions.Fraction):

- split: h is x truncated to 24 significant bits, |x - (h + l)| < 2^-46 |x| on the stated
  range, zeros, tiny values, infinities and NaNs as documented;
- join: the pair value to within one unit of the 53rd bit, for normalised and
  non-normalised pairs;
- add, sub, mul, multiply-accumulate: errors within small multiples of u^2 = 2^-48 of the
  operands' magnitudes (the error model the kernels' bounds rest on);
- division (the recomputed geometric factors' w / det): within 8 u^2 |x / y|;
- an 8-term dot product from binary64 inputs to within 8 2^-46 sum |a_j b_j|;
- the recomputed metric (kgeomdw.cuh: G = w |J| J^-1 J^-T, m = w |J| per node) against the
  oracle's binary64 factors, to within 64 u^2 of the node's largest G entry and of m.
The host build uses no contraction (-ffp-contract=off), as the device code uses
never-fused intrinsics.
"""
import ctypes
import os
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "dw_harness.cpp")
HDR = os.path.join(ROOT, "paper_1506_05996_gb300", "csrc", "kdw.cuh")
HDR2 = os.path.join(ROOT, "paper_1506_05996_gb300", "csrc", "kgeomdw.cuh")
OUT = os.path.join(ROOT, "paper_1506_05996_gb300", "_build", "dw_harness.so")
U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(map(os.path.getmtime, (SRC, HDR, HDR2))):
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", OUT, SRC],
                       check=True)
    return ctypes.CDLL(OUT)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def split(lib, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    h, l = np.zeros(len(x), np.float32), np.zeros(len(x), np.float32)
    lib.dwh_split(_p(x), _p(h), _p(l), ctypes.c_int64(len(x)))
    return h, l


def join(lib, h, l):
    h, l = np.ascontiguousarray(h, np.float32), np.ascontiguousarray(l, np.float32)
    y = np.zeros(len(h))
    lib.dwh_join(_p(h), _p(l), _p(y), ctypes.c_int64(len(h)))
    return y


def op(lib, k, xh, xl, yh, yl, ah=None, al=None):
    n = len(xh)
    ah = np.zeros(n, np.float32) if ah is None else ah.copy()
    al = np.zeros(n, np.float32) if al is None else al.copy()
    arrs = [np.ascontiguousarray(a, np.float32) for a in (xh, xl, yh, yl)]
    lib.dwh_op(ctypes.c_int(k), *[_p(a) for a in arrs], _p(ah), _p(al), ctypes.c_int64(n))
    return ah, al


def F(v):
    return Fr(float(v))


def rand_doubles(rng, n, lo=-60, hi=60):
    return rng.standard_normal(n) * np.exp2(rng.integers(lo, hi, n).astype(np.float64))


def rand_pairs(rng, n, lo=-40, hi=40):
    """normalised pairs of random binary64 values"""
    x = rand_doubles(rng, n, lo, hi)
    h = x.astype(np.float32)
    return h, (x - h.astype(np.float64)).astype(np.float32)


def test_split_truncates_to_24_and_47_bits(lib):
    rng = np.random.default_rng(1)
    x = rand_doubles(rng, 20000, -79, 126)
    x = x[(np.abs(x) >= 2.0 ** -80) & (np.abs(x) < 2.0 ** 127)]
    h, l = split(lib, x)
    for xi, hi, li in zip(x[:4000], h[:4000], l[:4000]):
        assert abs(F(xi) - F(hi) - F(li)) < Fr(2) ** -46 * abs(F(xi))
        # h is x truncated to 24 significant bits: same sign, |h| <= |x| < |h| + ulp(h)
        assert abs(F(hi)) <= abs(F(xi)) < abs(F(hi)) + Fr(float(np.spacing(np.float32(abs(hi)))))
        assert li == 0 or np.sign(li) == np.sign(xi)
    err = np.abs(x - (h.astype(np.float64) + l.astype(np.float64))) / np.abs(x)
    assert err.max() < 2.0 ** -46


def test_split_special_values(lib):
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-40, -1e-300, 2.0 ** -100, 3.0 * 2.0 ** -81,
                  2.0 ** 127 * 1.5, 2.0 ** 128, 1e300, 1.0, -1.0 - 2.0 ** -40])
    h, l = split(lib, x)
    assert h[0] == 0 and h[1] == 0 and np.signbit(h[1]) and l[0] == 0 and l[1] == 0
    assert h[2] == np.inf and h[3] == -np.inf and np.isnan(h[4])
    assert h[5] == 0 and h[6] == 0 and np.signbit(h[6])              # below binary32's range
    assert h[7] == np.float32(2.0 ** -100) and l[7] == 0               # exact; l below 2^-80 dropped
    assert h[8] == np.float32(3.0 * 2.0 ** -81) and l[8] == 0
    assert h[9] == np.float32(2.0 ** 127 * 1.5) and l[9] == 0
    assert h[10] == np.inf and h[11] == np.inf
    assert h[12] == 1.0 and l[12] == 0
    assert h[13] == -1.0 and l[13] == np.float32(-2.0 ** -40)


def test_join_is_the_pair_value(lib):
    rng = np.random.default_rng(2)
    h, l = rand_pairs(rng, 20000)
    y = join(lib, h, l)
    exact = h.astype(np.float64) + l.astype(np.float64)       # exact: at most 48 bits apart
    assert np.all(np.abs(y - exact) <= 2.0 ** -52 * np.abs(exact))
    # non-normalised pairs: l up to 2^10 ulp(h), either sign, and powers of two for h
    h2 = np.exp2(rng.integers(-30, 30, 5000)).astype(np.float32) * np.where(rng.random(5000) < .5, 1, -1)
    l2 = (h2 * rng.standard_normal(5000) * 2.0 ** -14).astype(np.float32)
    y2 = join(lib, h2, l2)
    for hi, li, yi in zip(h2[:3000], l2[:3000], y2[:3000]):
        ex = F(hi) + F(li)
        assert abs(F(yi) - ex) <= Fr(2) ** -52 * abs(ex)
    assert np.isnan(join(lib, np.array([np.nan]), np.array([0.0]))[0])
    assert join(lib, np.array([np.inf]), np.array([0.0]))[0] == np.inf
    assert join(lib, np.array([0.0]), np.array([0.0]))[0] == 0.0
    # split then join round trip
    x = rand_doubles(rng, 20000, -70, 120)
    x = x[np.abs(x) >= 2.0 ** -80]
    assert np.max(np.abs(join(lib, *split(lib, x)) - x) / np.abs(x)) < 2.0 ** -46


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_add_sub_mul_mac_error(lib, k):
    rng = np.random.default_rng(10 + k)
    n = 3000
    xh, xl = rand_pairs(rng, n, -20, 20)
    yh, yl = rand_pairs(rng, n, -20, 20)
    # half the cases nearly cancel (y close to -x)
    near = rng.random(n) < 0.5
    yh = np.where(near, -xh, yh)
    yl = np.where(near, (-xl * (1 + rng.standard_normal(n) * 1e-3)).astype(np.float32), yl)
    ah0, al0 = rand_pairs(rng, n, -20, 20)
    ah, al = op(lib, k, xh, xl, yh, yl, ah0, al0)
    for i in range(n):
        x, y = F(xh[i]) + F(xl[i]), F(yh[i]) + F(yl[i])
        got = F(ah[i]) + F(al[i])
        if k == 0:
            ex, mag = x + y, abs(x) + abs(y)
        elif k == 1:
            ex, mag = x - y, abs(x) + abs(y)
        elif k == 2:
            ex, mag = x * y, abs(x * y)
        else:
            a = F(ah0[i]) + F(al0[i])
            ex, mag = a + x * y, abs(a) + abs(x * y)
        assert abs(got - ex) <= Fr(4 * U2) * mag, (k, i)


def test_div_error(lib):
    """Quotient of two pairs: one reciprocal estimate of the divisor's head, the remainder
    x - q_h y formed with an exact product, one correction term (after Joldes, Muller and
    Popescu's pair division); its error stays within 8 u^2 of the quotient, for divisors with
    a large or a small tail and with head and tail of either sign."""
    rng = np.random.default_rng(21)
    n = 4000
    xh, xl = rand_pairs(rng, n, -20, 20)
    yh, yl = rand_pairs(rng, n, -20, 20)
    ah, al = op(lib, 4, xh, xl, yh, yl)
    for i in range(n):
        x, y = F(xh[i]) + F(xl[i]), F(yh[i]) + F(yl[i])
        q = x / y
        assert abs(F(ah[i]) + F(al[i]) - q) <= Fr(8 * U2) * abs(q), i
    # a power of two divides exactly; x / x is one to within 2 u^2 (the head of the quotient
    # may be 1 - u, the one-term correction then carries the rounded reciprocal's error)
    h, l = rand_pairs(rng, 50, -10, 10)
    two = np.full(50, 0.25, np.float32)
    qh, ql = op(lib, 4, h, l, two, np.zeros(50, np.float32))
    assert all(F(qh[i]) + F(ql[i]) == 4 * (F(h[i]) + F(l[i])) for i in range(50))
    qh, ql = op(lib, 4, h, l, h, l)
    assert all(abs(F(qh[i]) + F(ql[i]) - 1) <= Fr(2 * U2) for i in range(50))


def test_dot_product_from_binary64(lib):
    rng = np.random.default_rng(5)
    n, k = 2000, 8
    a, b = rng.standard_normal(n * k), rng.standard_normal(n * k) * 1e-3
    out = np.zeros(n)
    lib.dwh_dot(_p(a), _p(b), _p(out), ctypes.c_int64(n), ctypes.c_int(k))
    for i in range(n):
        ex = sum(F(a[i * k + j]) * F(b[i * k + j]) for j in range(k))
        mag = sum(abs(F(a[i * k + j]) * F(b[i * k + j])) for j in range(k))
        assert abs(F(out[i]) - ex) <= Fr(k * 2.0 ** -46) * mag


def _geom(lib, xe, t, rho, absolute=False):
    """The pair metric of one element at its p^3 nodes, as [6, i, j, k] and [i, j, k]."""
    p = len(t)
    phi = np.empty(2 * p)
    phi[0::2], phi[1::2] = (1 - t) / 2, (1 + t) / 2
    w3 = np.ascontiguousarray((rho[:, None, None] * rho[None, :, None] * rho[None, None, :]).transpose(2, 1, 0).ravel())
    G, m = np.zeros(6 * p ** 3), np.zeros(p ** 3)
    lib.dwh_geom(_p(np.ascontiguousarray(xe.ravel())), _p(phi), _p(w3), ctypes.c_int(p), ctypes.c_int(int(absolute)),
                 _p(G), _p(m))
    return G.reshape(6, p, p, p).transpose(0, 3, 2, 1), m.reshape(p, p, p).transpose(2, 1, 0)


def test_recomputed_metric_against_binary64(lib):
    """The pair metric that the recomputed-geometry FP64 operator evaluates per node, against
    the oracle's binary64 geometric factors (Sec. 2.3) of the same vertices: 30 elements of the
    32^3 lattice (+-20 %), n = 1..8, in place and moved 1000 units away.

    The reference takes the vertices relative to corner 0 (the same binary64 differences the
    pair code starts from), so it measures the pair arithmetic alone. The harness evaluates
    it as the kernel does: the corner sums once per line of nodes (i, j fixed), J completed per
    node. Bound: J's entries come from 4-term pair sums whose absolute terms add up to a few
    |J| on these elements, each step within a few u^2 of its terms; the cofactors, the
    determinant and the division multiply that by small condition numbers; the sums, J and the
    cofactors are renormalised before their products. Measured worst: 17 u^2 (G and m); 127
    and 65 u^2 without the renormalisation. A wrong sign, index or dropped term errs by O(1)."""
    from synth import lattice_hex_mesh
    from oracle.gll import gll_nodes_weights
    from oracle.geometry import geometric_factors
    mesh = lattice_hex_mesh(32, 0.2, 1)
    els = np.random.default_rng(7).choice(len(mesh.hex2vert), 30, replace=False)
    for shift in (0.0, 1000.0):
        for n in range(1, 9):
            t, rho = gll_nodes_weights(n)
            for e in els:
                xe = mesh.xyz[mesh.hex2vert[e]] + shift
                Gr, mr, _ = geometric_factors((xe - xe[0])[None], t, rho)
                G, m = _geom(lib, xe, t, rho)
                scale = np.abs(Gr[:, 0]).max(axis=0)
                assert np.all(np.abs(G - Gr[:, 0]) <= 64 * U2 * scale), (shift, n, e)
                assert np.all(np.abs(m - mr[0]) <= 64 * U2 * np.abs(mr[0])), (shift, n, e)


def test_recomputed_metric_needs_corner_relative_vertices(lib):
    """Why the element kernel stages its vertices relative to corner 0: summed from absolute
    coordinates 1000 units from the origin (|x| / h = 32,000), J loses about log2(32,000) = 15
    of the pairs' 48 bits, and the metric misses the bound above by orders of magnitude; the
    corner-relative form meets it (previous test)."""
    from synth import lattice_hex_mesh
    from oracle.gll import gll_nodes_weights
    from oracle.geometry import geometric_factors
    mesh = lattice_hex_mesh(32, 0.2, 1)
    t, rho = gll_nodes_weights(7)
    xe = mesh.xyz[mesh.hex2vert[5]] + 1000.0
    Gr, _, _ = geometric_factors((xe - xe[0])[None], t, rho)
    scale = np.abs(Gr[:, 0]).max(axis=0)
    G_abs, _ = _geom(lib, xe, t, rho, absolute=True)
    G_rel, _ = _geom(lib, xe, t, rho)
    assert np.max(np.abs(G_abs - Gr[:, 0]) / scale) > 4096 * U2
    assert np.max(np.abs(G_rel - Gr[:, 0]) / scale) <= 64 * U2
