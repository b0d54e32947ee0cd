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


def _small_problem():
    return Problem(lattice_hex_mesh(3, 0.2, 5), 3, 0.7, coarse_solver="exact")


def test_fpcg_without_correction_is_pcg():
    # fixed SPD P: z_k.r_k-1 = 0, so the Polak-Ribiere beta equals the one of Algorithm 1
    pr = _small_problem()
    b = pr.load(np.random.default_rng(3).standard_normal(pr.G))
    x0, it0, h0 = pr.solve(b, rtol=1e-10)[:3]
    x1, it1, h1, on = learned.fpcg(pr.apply_A, pr.apply_P, None, pr.mask, b, rtol=1e-10)
    assert it1 == it0 and on == 0
    np.testing.assert_allclose(h1, h0, rtol=1e-6, atol=1e-13)
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-9 * np.abs(x0).max())


def test_fpcg_with_exact_correction_ends_in_one_step():
    # N = A^-1 on the free DOFs makes P r + N(r - A P r) = A^-1 r
    pr = _small_problem()
    A = pr.assembled().toarray()
    free = pr.mask == 0
    Aff = A[np.ix_(free, free)]
    def exact(v):
        out = np.zeros_like(v)
        out[free] = np.linalg.solve(Aff, v[free])
        return out
    b = pr.load(np.random.default_rng(4).standard_normal(pr.G))
    x, it, hist, on = learned.fpcg(pr.apply_A, pr.apply_P, exact, pr.mask, b, rtol=1e-10)
    assert it == 1 and on == 1 and hist[-1] < 1e-11


def test_fpcg_stall_switches_correction_off():
    pr = _small_problem()
    b = pr.load(np.random.default_rng(5).standard_normal(pr.G))
    rng = np.random.default_rng(6)
    noise = lambda v: rng.standard_normal(v.shape) * np.linalg.norm(v) * (pr.mask == 0)
    x, it, hist, on = learned.fpcg(pr.apply_A, pr.apply_P, noise, pr.mask, b, rtol=1e-8, maxit=400, theta=-1e300)
    assert hist[-1] <= 1e-8 and on < it
    ref_it = pr.solve(b, rtol=1e-8)[1]
    assert it <= ref_it + on + 10


def test_training_pair_satisfies_A_delta_equals_s():
    pr = _small_problem()
    A = pr.assembled().toarray()
    free = pr.mask == 0
    rng = np.random.default_rng(7)
    b = pr.load(rng.standard_normal(pr.G))
    x_star = np.zeros(pr.G)
    x_star[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    x_k = pr.solve(b, rtol=1e-8, maxit=3)[0]
    s, delta, r, z0 = learned.training_pair(pr.apply_A, pr.apply_P, pr.mask, b, x_star, x_k)
    np.testing.assert_allclose(pr.apply_A(delta), s, atol=1e-10 * np.abs(s).max())
    np.testing.assert_allclose(pr.apply_A(delta + z0), r, atol=1e-10 * np.abs(r).max())
    assert np.all(s[~free] == 0) and np.all(delta[~free] == 0)


def test_energy_loss_is_energy_norm_ratio_and_gradient_is_exact():
    pr = _small_problem()
    A = pr.assembled().toarray()
    free = pr.mask == 0
    rng = np.random.default_rng(9)
    delta = rng.standard_normal(pr.G) * free
    v = np.where(free, A @ delta, 0.0)
    theta = rng.standard_normal(learned.n_params()) * 0.2
    args = (pr.apply_A, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    loss, g = learned.energy_loss_and_grad(theta, v, delta, *args)
    c = learned.correction(theta, v, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    d = delta - c
    assert abs(loss - (d @ A @ d) / (delta @ A @ delta)) <= 1e-10 * loss
    zero = theta.copy()
    W3, b3 = learned.unpack(zero)[2]
    W3[...] = 0.0
    b3[...] = 0.0
    assert abs(learned.energy_loss_and_grad(zero, v, delta, *args)[0] - 1.0) < 1e-12
    for i in rng.choice(theta.size, 12, replace=False):
        e = np.zeros_like(theta)
        e[i] = 1e-6
        fd = (learned.energy_loss_and_grad(theta + e, v, delta, *args)[0]
              - learned.energy_loss_and_grad(theta - e, v, delta, *args)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_angle_loss_is_line_search_energy_and_gradient_is_exact():
    pr = _small_problem()
    A = pr.assembled().toarray()
    free = pr.mask == 0
    rng = np.random.default_rng(10)
    b = pr.load(rng.standard_normal(pr.G))
    x_star = np.zeros(pr.G)
    x_star[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    x_k = pr.solve(b, rtol=1e-8, maxit=2)[0]
    s, delta, r, z0 = learned.training_pair(pr.apply_A, pr.apply_P, pr.mask, b, x_star, x_k)
    theta = rng.standard_normal(learned.n_params()) * 0.2
    args = (pr.apply_A, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    loss, g = learned.angle_loss_and_grad(theta, s, r, z0, delta, *args)
    z = z0 + learned.correction(theta, s, pr.m_N, pr.l2g, pr.h, pr.lam, pr.mask)
    e = x_star - x_k
    alpha = (z @ A @ e) / (z @ A @ z)                      # exact line search along z
    left = (e - alpha * z) @ A @ (e - alpha * z) / (e @ A @ e)
    assert abs(1.0 - (1.0 - loss) ** 2 - left) <= 1e-9
    assert (loss < 1.0) == (z @ A @ e > 0)
    for i in rng.choice(theta.size, 12, replace=False):
        d = np.zeros_like(theta)
        d[i] = 1e-6
        fd = (learned.angle_loss_and_grad(theta + d, s, r, z0, delta, *args)[0]
              - learned.angle_loss_and_grad(theta - d, s, r, z0, delta, *args)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_fpcg_safeguard_rejects_a_correction_that_cancels_descent():
    pr = _small_problem()
    b = pr.load(np.random.default_rng(11).standard_normal(pr.G))
    # a correction c = -2 z0 turns every step into an ascent direction: always rejected
    last = {}

    def P(r):
        last["z"] = pr.apply_P(r)
        return last["z"]

    flip = lambda v: -2.0 * last["z"]
    x, it, hist, on = learned.fpcg(pr.apply_A, P, flip, pr.mask, b, rtol=1e-10, window=0)
    ref = pr.solve(b, rtol=1e-10)
    assert on == 0 and it == ref[1]


def test_correction_abs_bounds_and_equals_the_positive_network():
    """oracle.learned.correction_abs (the network with |W|, |b|, |features| and no ReLU,
    scaled and averaged like the correction) bounds |N(v)| at every node, and equals N(v)
    when the weights, biases and features are all nonnegative (every ReLU is then the
    identity)."""
    from oracle.learned import correction, correction_abs, n_params
    from oracle.problem import Problem
    from synth import lattice_hex_mesh
    pr = Problem(lattice_hex_mesh(2, 0.2, 3), 3, 0.7, coarse_solver=None, with_schwarz=False)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(n_params()) * 0.3
    v = rng.standard_normal(pr.G) * (pr.mask == 0)
    c = correction(theta, v, pr.m_N, pr.l2g, pr.h if hasattr(pr, "h") else _boxes(pr), pr.lam, pr.mask)
    ca = correction_abs(theta, v, pr.m_N, pr.l2g, pr.h if hasattr(pr, "h") else _boxes(pr), pr.lam, pr.mask)
    assert np.all(np.abs(c) <= ca * (1 + 1e-12) + 1e-300)
    assert np.max(np.abs(c) / np.where(ca > 0, ca, 1.0)) < 1.0
    tpos = np.abs(theta)
    vpos = np.abs(v)
    h = pr.h if hasattr(pr, "h") else _boxes(pr)
    cp = correction(tpos, vpos, pr.m_N, pr.l2g, h, pr.lam, pr.mask)
    cpa = correction_abs(tpos, vpos, pr.m_N, pr.l2g, h, pr.lam, pr.mask)
    np.testing.assert_allclose(cp, cpa, rtol=1e-12, atol=0)


def _boxes(pr):
    from oracle.geometry import element_box_sizes
    return element_box_sizes(pr.xyz_e)
