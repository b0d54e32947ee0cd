"""Training and evaluation of the learned correction (not in the paper).

The network (include/sem.h, sem_net_*) adds N(r - A P r) to the two-scale preconditioner
inside flexible PCG. Its training pairs come from the solver itself: on each training
problem a converged solve gives x*, solves stopped after k iterations give iterates x_k,
and sem_net_pair turns each (x*, x_k) into the network input s = r - A P r and the target
delta = x* - x_k - P r. Training runs the library's own BF16 forward/backward kernels and
Adam (sem_net_train_step). Everything here is orchestration of library calls; the only
arithmetic outside the library is forming the load vector b = m_N s(x_N) from the
synthetic input.
"""
import math
import time

import numpy as np
import torch

from synth import gaussian_load, lattice_hex_mesh, manufactured_s
from .sem import (SEM_GEOM_RECOMPUTE, SemProblem, sem_learned_iterations, sem_net_create, sem_net_destroy,
                  sem_net_pair, sem_net_train_step, sem_set_learned)


def make_problem(E, a, seed, n, lam, load="manufactured", geom="stored", mixed=False, load_seed=0):
    """A seeded lattice problem and its load vector b (masked)."""
    mesh = lattice_hex_mesh(E, a, seed)
    prob = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom=geom, mixed=mixed)
    free = (prob.mask() == 0).to(torch.float64)
    if load == "manufactured":
        X = prob.dof_coords().cpu().numpy()
        s = torch.as_tensor(manufactured_s(X, lam), device="cuda")
        b = prob.mass() * s * free
    else:
        b = torch.as_tensor(gaussian_load(prob.n_dof, load_seed), device="cuda") * free
    return prob, b.contiguous()


def harvest(prob, b, ks=(0, 1, 2, 4, 8, 16), net=None):
    """Training samples (s, delta, r, z0) at the iterates x_k (k in ks, below convergence) of
    PCG, or of the flexible PCG with `net` attached (samples from the solver's own path)."""
    sem_set_learned(prob.h, None)
    xs, _, it, _, _ = prob.solve(b, rtol=1e-11, maxit=2000)
    sem_set_learned(prob.h, net)
    out = []
    for k in ks:
        if k >= it:
            break
        xk = prob.solve(b, rtol=0.0, maxit=k)[0] if k > 0 else torch.zeros_like(b)
        vecs = [torch.empty_like(b) for _ in range(4)]
        sem_net_pair(prob.h, b, xs, xk, *vecs)
        out.append(tuple(vecs))
    sem_set_learned(prob.h, None)
    return out


def training_set(n_meshes, E, n, a=0.2, lam_max=10.0, seed=0, ks=(0, 1, 2, 4, 8, 16)):
    """Seeded training problems: E^3 hexes, order n, lambda ~ U[0, lam_max], alternating a
    manufactured and a Gaussian load; returns (problems with their loads, samples
    [(problem, s, delta, r, z0)])."""
    rng = np.random.default_rng(seed)
    problems, samples = [], []
    for m in range(n_meshes):
        lam = float(rng.uniform(0.0, lam_max))
        prob, b = make_problem(E, a, 1000 + seed * 100000 + m, n, lam, geom="recompute",
                               load="manufactured" if m % 2 == 0 else "gaussian", load_seed=77 + m)
        problems.append((prob, b))
        samples += [(prob,) + v for v in harvest(prob, b, ks)]
    return problems, samples


def train(net, samples, steps, lr=1e-3, seed=0, loss="angle"):
    """Adam steps on randomly drawn samples with a cosine learning-rate decay; the losses."""
    rng = np.random.default_rng(seed)
    losses = []
    for t in range(steps):
        prob, s, d, r, z0 = samples[int(rng.integers(len(samples)))]
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * t / steps))
        losses.append(sem_net_train_step(net, prob.h, s, d, lr_t, loss, r, z0))
    return losses


def timed_solve(prob, b, net, rtol=1e-8, maxit=2000, reps=1, window=8, ratio=0.5, theta=0.25):
    """(iterations, seconds per solve, true relative residual, status, iterations that used the
    correction) with the network attached or not."""
    sem_set_learned(prob.h, net, window, ratio, theta)
    x = torch.empty_like(b)
    prob.solve(b, rtol=rtol, maxit=maxit, x=x)      # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, rc, it, _, tr = prob.solve(b, rtol=rtol, maxit=maxit, x=x)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    used = sem_learned_iterations(prob.h)
    sem_set_learned(prob.h, None)
    return it, dt, tr, rc, used


__all__ = ["make_problem", "harvest", "training_set", "train", "timed_solve", "sem_net_create",
           "sem_net_destroy", "SEM_GEOM_RECOMPUTE"]
