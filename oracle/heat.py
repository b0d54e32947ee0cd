"""Heat equation by backward Euler (Sec. 5, heat-equation experiment), FP64.

Test infrastructure only (like the rest of oracle/): never imported by the library.

The model problem c u - div(kappa grad u) = s with c = 1/dt and s = u_prev/dt + Q/(rho c_p)
is, divided by kappa, the library's operator with lambda = 1/(kappa dt):
    A u = M (lambda u_prev + g),   g = Q / (rho c_p kappa),
A the (masked) SEM operator with that lambda and M the lumped GLL mass. One step is that
linear solve, written here with a sparse direct solve of the assembled matrix.

Pinned by: without a mask and with g = 0 a constant field stays constant (K 1 = 0); without
a mask the total heat obeys 1^T M u = 1^T M u_prev + (1 / lambda) 1^T M g exactly; with a
Dirichlet mask and g = 0 the M-norm never grows.
"""
import numpy as np
from scipy.sparse.linalg import splu


class HeatStepper:
    def __init__(self, problem):
        self.pr = problem
        self.lu = splu(problem.assembled().tocsc())

    def rhs(self, u_prev, g):
        pr = self.pr
        return np.where(pr.mask > 0, 0.0, pr.m_N * (pr.lam * u_prev + g))

    def step(self, u_prev, g):
        return self.lu.solve(self.rhs(u_prev, g))
