"""Shared helpers of the GPU parity tests: a library problem and the oracle on the
same seeded mesh, with the DOF permutation between them found by position."""
import numpy as np
import torch

from oracle.problem import Problem
from paper_1506_05996_gb300.sem import SemProblem


class Pair:
    def __init__(self, mesh, n, lam, geom="stored", neumann=False, coarse=True, schwarz=True, kcycle=False):
        self.gpu = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom=geom, neumann=neumann)
        if kcycle:
            self.gpu.set_coarse_solver("kcycle")
        self.ref = Problem(mesh, n, lam, dirichlet=not neumann,
                           coarse_solver=("kcycle" if kcycle else "amg") if coarse else None, with_schwarz=schwarz)
        self._match()

    def _match(self):
        X = self.gpu.dof_coords().cpu().numpy()
        oi = np.lexsort(np.round(self.ref.coords, 9).T)
        gi = np.lexsort(np.round(X, 9).T)
        perm = np.empty_like(gi)
        perm[oi] = gi                       # oracle dof k  <->  gpu dof perm[k]
        assert np.abs(X[perm] - self.ref.coords).max() < 1e-12
        self.perm = perm
        self.perm_t = torch.as_tensor(perm, device="cuda")

    def to_gpu(self, v):
        out = torch.zeros(self.gpu.n_dof, dtype=torch.float64, device="cuda")
        out[self.perm_t] = torch.as_tensor(np.ascontiguousarray(v), device="cuda")
        return out

    def to_ref(self, t):
        return t.cpu().numpy()[self.perm]


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# History tolerances of the solve parity tests. The recursive residual r_k = r_k-1 - alpha A p
# carries the operator's rounding of every iteration, measured against ||b||. The
# double-FP32 element kernels of SEM_PREC_FP64 round at 2^-46 of their operands'
# magnitudes where binary64 rounds at 2^-53, so in that arithmetic the absolute tolerance of
# a history entry is 2^7 times the binary64 one (SEM_PREC_FP64_NATIVE keeps the latter).
DW_HIST_SCALE = 2.0 ** 7


def hist_atol(base, prec="fp64"):
    return base * (DW_HIST_SCALE if prec == "fp64" else 1.0)
