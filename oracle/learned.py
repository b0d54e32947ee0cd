"""Learned correction: a per-element 3D convolutional network (FP64 reference).

Not in the paper. The network adds a correction N(r) to the two-scale preconditioner
inside flexible PCG (z = P r + N(r)). Definition used by the oracle and, independently
written, by the GPU kernels:

  features of element e on its (n+1)^3 GLL grid (channel, node):
    hbar = (hx + hy + hz) / 3, s_l = (r_N / m_N) hbar^2 at the node's DOF N,
    sigma_e = sqrt(mean_l s_l^2) + 1e-300,
    c0 = s_l / sigma_e, c1 = hx / hbar, c2 = hy / hbar, c3 = hz / hbar,
    c4 = lambda hbar^2 / (1 + lambda hbar^2)           (c1..c4 constant over the element)
  network: conv3x3x3(5 -> 8) + ReLU, conv3x3x3(8 -> 8) + ReLU, conv3x3x3(8 -> 1); every
    convolution is a correlation with zero padding on the element grid, bias per channel;
  output: local correction c_l = y_l sigma_e; global correction = average of c_l over the
    local copies of each DOF, zero on Dirichlet DOFs.
  training loss for one sample: mean over all local nodes of (y_l - t_l / sigma_e)^2, t the
    local target correction.

Pinned by: single-channel convolution = scipy.ndimage.correlate (constant 0 mode), and the
backward pass = central finite differences of the loss in FP64.
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
