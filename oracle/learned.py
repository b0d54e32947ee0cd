"""Learned correction: a per-element 3D convolutional network (FP64 reference).

Test infrastructure only (like the rest of oracle/): never imported by the library.

Not in the paper. The network corrects what the two-scale preconditioner leaves: inside
flexible PCG, z = P r + N(r - A P r), with the Polak-Ribiere form of the CG beta,
beta_k = z_k.(r_k - r_k-1) / (z_k-1.r_k-1), and the correction switched off for the rest
of a solve at the first iteration k >= W with ||r_k|| >= ratio ||r_k-W|| (W = 0: never;
W = 8, ratio = 0.5 by default). Training pairs
from an iterate x_k of A x = b with solution x*: r = b - A x_k, z0 = P r, input
s = r - A z0, target delta = x* - x_k - z0 (so A delta = s). Definition used by the
oracle and, independently written, by the GPU kernels:

  features of element e on its (n+1)^3 GLL grid (channel, node):
    hbar = (hx + hy + hz) / 3, s_l = (r_N / m_N) hbar^2 at the node's DOF N,
    sigma_e = sqrt(mean_l s_l^2) + 1e-300,
    c0 = s_l / sigma_e, c1 = hx / hbar, c2 = hy / hbar, c3 = hz / hbar,
    c4 = lambda hbar^2 / (1 + lambda hbar^2)           (c1..c4 constant over the element)
  network: conv3x3x3(5 -> 8) + ReLU, conv3x3x3(8 -> 8) + ReLU, conv3x3x3(8 -> 1); every
    convolution is a correlation with zero padding on the element grid, bias per channel;
  output: local correction c_l = y_l sigma_e; global correction = average of c_l over the
    local copies of each DOF, zero on Dirichlet DOFs.
  training losses for one sample (input v, target delta):
    "l2":     mean over all local nodes of (y_l - t_l / sigma_e)^2, t the local target;
    "energy": L(c) = 1 + (c^T A c - 2 c^T v) / (delta^T v) for the global correction c,
              which equals ||delta - c||_A^2 / ||delta||_A^2 when v = A delta (the norm CG
              minimises); dL/dc = -2 (v - A c) / (delta^T v) on the free DOFs.
    "angle":  with the pair's residual r and z0 = P r, z = z0 + c and e = delta + z0 (so
              A e = r): L(c) = 1 - z^T r / sqrt((z^T A z)(e^T r)) = 1 - cos of the A-angle
              between z and e (1 - (1 - L)^2 is the share of ||e||_A^2 left after an exact
              line search along z); invariant to positive scaling of z, and it rewards the
              orientation descent needs. A z = r - q with q = v - A c (since A z0 = r - v);
              dL/dc = -(r - (a / Q) A z) / sqrt(Q E), a = z^T r, Q = z^T A z, E = e^T r.
  safeguard inside flexible PCG: the correction is used in an iteration only if
    (z0 + c)^T r >= theta z0^T r (theta = 0.25 by default), else that iteration takes z0.

Pinned by: single-channel convolution = scipy.ndimage.correlate (constant 0 mode); the
backward pass = central finite differences of the loss in FP64 (both losses); the energy
loss equals ||delta - c||_A^2 / ||delta||_A^2 from the assembled matrix when v = A delta,
and is 1 for a zero network; the angle loss gives 1 - cos of the A-angle between z and the
exact error (assembled matrix, direct solve, exact line search); flexible PCG with N = 0
takes the iterations of plain PCG (for a fixed SPD P, z_k.r_k-1 = 0, so the Polak-Ribiere
beta equals Algorithm 1's); with N = A^-1 (dense solve) the composed preconditioner is
A^-1 and the solve ends after one iteration; a training pair satisfies A delta = s.
"""
import numpy as np

LAYERS = [(5, 8, True), (8, 8, True), (8, 1, False)]   # (in, out, relu)


def n_params():
    return sum(co * ci * 27 + co for ci, co, _ in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W [co, ci, 3, 3, 3], b [co])] (layer order, W then b)."""
    out, k = [], 0
    for ci, co, _ in LAYERS:
        W = theta[k:k + co * ci * 27].reshape(co, ci, 3, 3, 3)
        k += co * ci * 27
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    return out


def conv3d(x, W, b):
    """y[e, co, i, j, k] = b[co] + sum_{ci, a, c, d} W[co, ci, a, c, d] x[e, ci, i+a-1, j+c-1, k+d-1]."""
    E, ci, p = x.shape[0], x.shape[1], x.shape[2]
    xp = np.zeros((E, ci, p + 2, p + 2, p + 2))
    xp[:, :, 1:p + 1, 1:p + 1, 1:p + 1] = x
    y = np.zeros((E, W.shape[0], p, p, p)) + b[None, :, None, None, None]
    for a in range(3):
        for c in range(3):
            for d in range(3):
                y += np.einsum("oi,eijkl->eojkl", W[:, :, a, c, d], xp[:, :, a:a + p, c:c + p, d:d + p])
    return y


def conv3d_backward(x, W, gy):
    """Gradients of sum(gy * conv3d(x, W, b)) with respect to x, W and b."""
    E, ci, p = x.shape[0], x.shape[1], x.shape[2]
    xp = np.zeros((E, ci, p + 2, p + 2, p + 2))
    xp[:, :, 1:p + 1, 1:p + 1, 1:p + 1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for a in range(3):
        for c in range(3):
            for d in range(3):
                gW[:, :, a, c, d] = np.einsum("eojkl,eijkl->oi", gy, xp[:, :, a:a + p, c:c + p, d:d + p])
                gxp[:, :, a:a + p, c:c + p, d:d + p] += np.einsum("oi,eojkl->eijkl", W[:, :, a, c, d], gy)
    gb = gy.sum(axis=(0, 2, 3, 4))
    return gxp[:, :, 1:p + 1, 1:p + 1, 1:p + 1], gW, gb


def forward(theta, x):
    """Network output y [E, 1, p, p, p] and the cache of layer inputs / pre-activations."""
    cache = []
    h = x
    for (W, b), (_, _, relu) in zip(unpack(theta), LAYERS):
        z = conv3d(h, W, b)
        cache.append((h, z))
        h = np.maximum(z, 0.0) if relu else z
    return h, cache


def backward(theta, cache, gy):
    """Gradient of sum(gy * y) with respect to the flat parameters."""
    grads = []
    g = gy
    for (W, b), (h, z), (_, _, relu) in zip(reversed(unpack(theta)), reversed(cache), reversed(LAYERS)):
        if relu:
            g = g * (z > 0)
        gx, gW, gb = conv3d_backward(h, W, g)
        grads.append((gW, gb))
        g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.ravel(), gb]
    return np.concatenate(flat)


def features(r, m_N, l2g, h, lam):
    """Input channels [E, 5, p, p, p] and sigma [E] from a global residual r."""
    hbar = h.mean(axis=1)
    s = (r / m_N)[l2g] * (hbar ** 2)[:, None, None, None]
    sigma = np.sqrt(np.mean(s.reshape(s.shape[0], -1) ** 2, axis=1)) + 1e-300
    E, p = l2g.shape[0], l2g.shape[1]
    x = np.zeros((E, 5, p, p, p))
    x[:, 0] = s / sigma[:, None, None, None]
    x[:, 1] = (h[:, 0] / hbar)[:, None, None, None]
    x[:, 2] = (h[:, 1] / hbar)[:, None, None, None]
    x[:, 3] = (h[:, 2] / hbar)[:, None, None, None]
    q = lam * hbar ** 2
    x[:, 4] = (q / (1.0 + q))[:, None, None, None]
    return x, sigma


def correction(theta, r, m_N, l2g, h, lam, mask):
    """Global correction N(r): local outputs times sigma, averaged over the copies of each DOF."""
    x, sigma = features(r, m_N, l2g, h, lam)
    y, _ = forward(theta, x)
    c = y[:, 0] * sigma[:, None, None, None]
    G = m_N.shape[0]
    tot = np.bincount(l2g.ravel(), weights=c.ravel(), minlength=G)
    cnt = np.bincount(l2g.ravel(), minlength=G)
    out = tot / cnt
    return np.where(mask > 0, 0.0, out)


def energy_loss_and_grad(theta, v, delta, apply_A, m_N, l2g, h, lam, mask):
    """Energy loss of the global correction c = N(v) and its parameter gradient."""
    x, sigma = features(v, m_N, l2g, h, lam)
    y, cache = forward(theta, x)
    G = m_N.shape[0]
    free = mask == 0
    cnt = np.bincount(l2g.ravel(), minlength=G)
    c = np.bincount(l2g.ravel(), weights=(y[:, 0] * sigma[:, None, None, None]).ravel(), minlength=G) / cnt
    c = np.where(free, c, 0.0)
    q = np.where(free, v - apply_A(c), 0.0)
    den = delta @ v
    loss = 1.0 - c @ (v + q) / den
    dc = np.where(free, -2.0 * q / den, 0.0)           # dL/dc
    gy = (dc / cnt)[l2g] * sigma[:, None, None, None]  # dc_N / dy_l = sigma_e / multiplicity
    return loss, backward(theta, cache, gy[:, None])


def angle_loss_and_grad(theta, v, r, z0, delta, apply_A, m_N, l2g, h, lam, mask):
    """Angle loss of z = z0 + N(v) against the error e = delta + z0, and its parameter gradient."""
    x, sigma = features(v, m_N, l2g, h, lam)
    y, cache = forward(theta, x)
    G = m_N.shape[0]
    free = mask == 0
    cnt = np.bincount(l2g.ravel(), minlength=G)
    c = np.bincount(l2g.ravel(), weights=(y[:, 0] * sigma[:, None, None, None]).ravel(), minlength=G) / cnt
    c = np.where(free, c, 0.0)
    q = np.where(free, v - apply_A(c), 0.0)
    z = z0 + c
    Az = r - q
    a, Q, E = z @ r, z @ Az, (delta + z0) @ r
    loss = 1.0 - a / np.sqrt(Q * E)
    dc = np.where(free, -(r - (a / Q) * Az) / np.sqrt(Q * E), 0.0)
    gy = (dc / cnt)[l2g] * sigma[:, None, None, None]
    return loss, backward(theta, cache, gy[:, None])


def loss_and_grad(theta, r, target_local, m_N, l2g, h, lam):
    """Training loss (mean over local nodes of (y - t/sigma)^2) and its parameter gradient."""
    x, sigma = features(r, m_N, l2g, h, lam)
    y, cache = forward(theta, x)
    t = target_local / sigma[:, None, None, None]
    d = y[:, 0] - t
    L = d.size
    loss = np.sum(d ** 2) / L
    gy = (2.0 / L) * d[:, None]
    return loss, backward(theta, cache, gy)




def training_pair(apply_A, apply_P, mask, b, x_star, x_k):
    """(s, delta, r, z0): r = b - A x_k, z0 = P r, s = r - A z0, delta = x* - x_k - z0 (0 on masked DOFs)."""
    free = mask == 0
    r = np.where(free, b - apply_A(x_k), 0.0)
    z0 = apply_P(r)
    s = np.where(free, r - apply_A(z0), 0.0)
    delta = np.where(free, x_star - x_k - z0, 0.0)
    return s, delta, r, z0


def fpcg(apply_A, apply_P, correction, mask, b, rtol=1e-8, maxit=1000, window=8, ratio=0.5, theta=0.25):
    """Flexible PCG with z = P r + correction(r - A P r); correction None = plain P.

    Returns (x, iterations, relative residual history, iterations that used the correction).
    """
    free = mask == 0
    r = np.where(free, b, 0.0)
    x = np.zeros_like(r)
    r_prev = np.zeros_like(r)
    bb = r @ r
    hist = [1.0 if bb > 0 else 0.0]
    if bb == 0.0:
        return x, 0, np.array(hist), 0
    on = correction is not None
    on_iters = 0
    rrs = [bb]
    p = None
    rz_old = None
    for k in range(1, maxit + 1):
        z = apply_P(r)
        if on:
            c = correction(np.where(free, r - apply_A(z), 0.0))
            if (z + c) @ r >= theta * (z @ r):
                z = z + c
                on_iters += 1
        rz = z @ r
        p = z.copy() if p is None else z + ((rz - z @ r_prev) / rz_old) * p
        rz_old = rz
        f = apply_A(p)
        alpha = rz / (p @ f)
        x = x + alpha * p
        r_prev = r
        r = r - alpha * f
        rr = r @ r
        rrs.append(rr)
        if on and window > 0 and k >= window and rr >= ratio ** 2 * rrs[k - window]:
            on = False
        hist.append(np.sqrt(rr / bb))
        if hist[-1] <= rtol:
            return x, k, np.array(hist), on_iters
    return x, maxit, np.array(hist), on_iters


def correction_abs(theta, v, m_N, l2g, h, lam, mask):
    """Magnitude of every term of the network's correction: the same evaluation with |W|, |b|
    and |features| and no ReLU (|ReLU(a)| <= |a|), times sigma_e, averaged over the local
    copies like the correction itself. Rounding bounds of a reduced-precision evaluation are
    multiples of this vector (each layer's sum errs by at most gamma_K times the sum of its
    terms' magnitudes, and such errors pass the next layers' |W| unchanged in sign)."""
    feats, sigma = features(v, m_N, l2g, h, lam)
    x = np.abs(feats)
    for W, b in unpack(theta):
        x = conv3d(x, np.abs(W), np.abs(b))
    c_loc = x[:, 0] * sigma[:, None, None, None]
    G = m_N.shape[0]
    cnt = np.bincount(l2g.ravel(), minlength=G).astype(np.float64)
    tot = np.bincount(l2g.ravel(), weights=c_loc.ravel(), minlength=G)
    out = tot / np.where(cnt > 0, cnt, 1.0)
    return np.where(mask > 0, 0.0, out)
