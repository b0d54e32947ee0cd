"""Pins for oracle/heat.py (backward-Euler heat steps, Sec. 5)."""
import numpy as np

from oracle.heat import HeatStepper
from oracle.problem import Problem
from synth import lattice_hex_mesh, moving_source


def _rod(neumann, lam=40.0):
    return Problem(lattice_hex_mesh((2, 2, 5), 0.2, 5, box=(1.0, 1.0, 2.5)), 3, lam,
                   dirichlet=not neumann, coarse_solver=None, with_schwarz=False)


def test_constant_field_is_steady_without_mask():
    pr = _rod(neumann=True)
    hs = HeatStepper(pr)
    u = np.full(pr.G, 3.25)
    np.testing.assert_allclose(hs.step(u, np.zeros(pr.G)), u, rtol=1e-12)


def test_total_heat_balance_without_mask():
    pr = _rod(neumann=True)
    hs = HeatStepper(pr)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(pr.G)
    for k in range(3):
        g = moving_source(pr.coords, 0.1 * k, width=0.4)
        u_new = hs.step(u, g)
        assert abs(pr.m_N @ u_new - (pr.m_N @ u + (pr.m_N @ g) / pr.lam)) <= 1e-11 * (abs(pr.m_N @ u) + 1.0)
        u = u_new


def test_mass_norm_decays_with_dirichlet_and_no_source():
    pr = _rod(neumann=False)
    hs = HeatStepper(pr)
    u = np.random.default_rng(2).standard_normal(pr.G) * (pr.mask == 0)
    prev = np.sqrt(u @ (pr.m_N * u))
    for _ in range(4):
        u = hs.step(u, np.zeros(pr.G))
        cur = np.sqrt(u @ (pr.m_N * u))
        assert cur < prev
        prev = cur
