"""Pins for oracle/learned.py (the learned-correction network; not in the paper)."""
import numpy as np
import scipy.ndimage

from oracle import learned
from synth import lattice_hex_mesh
from oracle.problem import Problem


def test_conv_is_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 1, 6, 6, 6))
    W = rng.standard_normal((1, 1, 3, 3, 3))
    y = learned.conv3d(x, W, np.array([0.25]))
    ref = scipy.ndimage.correlate(x[0, 0], W[0, 0], mode="constant", cval=0.0) + 0.25
    np.testing.assert_allclose(y[0, 0], ref, atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(learned.n_params()) * 0.3
    x = rng.standard_normal((2, 5, 4, 4, 4))
    gy = rng.standard_normal((2, 1, 4, 4, 4))
    y, cache = learned.forward(theta, x)
    g = learned.backward(theta, cache, gy)
    f = lambda th: np.sum(gy * learned.forward(th, x)[0])
    idx = rng.choice(theta.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = eps
        fd = (f(theta + e) - f(theta - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_gradient_and_correction_properties():
    pr = Problem(lattice_hex_mesh(2, 0.2, 3), 3, 1.0, coarse_solver=None)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(pr.G) * (pr.mask == 0)
    theta = rng.standard_normal(learned.n_params()) * 0.2
    t = rng.standard_normal(pr.l2g.shape)
    loss, g = learned.loss_and_grad(theta, r, t, pr.m_N, pr.l2g, pr.h, pr.lam)
    i = 7
    e = np.zeros_like(theta)
    e[i] = 1e-6
    lp = learned.loss_and_grad(theta + e, r, t, pr.m_N, pr.l2g, pr.h, pr.lam)[0]
    lm = learned.loss_and_grad(theta - e, r, t, pr.m_N, pr.l2g, pr.h, pr.lam)[0]
    assert abs((lp - lm) / 2e-6 - g[i]) < 1e-6 * max(1.0, abs(g[i]))
    c = learned.correction(theta, r, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    assert np.all(c[pr.mask > 0] == 0)
    # scale equivariance: N(a r) = a N(r) for a > 0 (features are normalised per element)
    c2 = learned.correction(theta, 3.5 * r, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    np.testing.assert_allclose(c2, 3.5 * c, rtol=1e-12, atol=1e-300)
