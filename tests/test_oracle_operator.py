"""Pins for oracle/operator.py (Eq. R, Algorithm 2, explicit assembly)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from synth import lattice_hex_mesh, HexMesh, manufactured_u, manufactured_s
from oracle.problem import Problem

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.2, 1.1]])


def sheared(E, seed=0):
    m = lattice_hex_mesh(E, 0.0, seed)
    return HexMesh(xyz=m.xyz @ SHEAR.T + 0.5, hex2vert=m.hex2vert)


@pytest.mark.parametrize("E,n,lam,a", [(1, 3, 0.0, 0.2), (2, 3, 1.3, 0.2), (2, 4, 0.0, 0.1),
                                       (4, 3, 0.0, 0.1), (2, 2, 2.0, 0.2)])
def test_matfree_equals_assembled(E, n, lam, a):
    m = lattice_hex_mesh(E, a, 7)
    for dirichlet in (False, True):
        pr = Problem(m, n, lam, dirichlet=dirichlet, coarse_solver=None, with_schwarz=False)
        A = pr.assembled()
        x = np.random.default_rng(1).standard_normal(pr.G)
        y1, y2 = pr.apply_A(x), A @ x
        assert np.max(np.abs(y1 - y2)) <= 1e-13 * np.max(np.abs(y2))


def test_symmetry_and_constant_nullspace():
    m = lattice_hex_mesh(3, 0.2, 8)
    for lam in (0.0, 1.7):
        pr = Problem(m, 4, lam, dirichlet=False, coarse_solver=None, with_schwarz=False)
        rng = np.random.default_rng(2)
        x, y = rng.standard_normal(pr.G), rng.standard_normal(pr.G)
        Ax, Ay = pr.apply_A(x), pr.apply_A(y)
        assert abs(y @ Ax - x @ Ay) < 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)
        one = pr.apply_A(np.ones(pr.G))
        np.testing.assert_allclose(one, lam * pr.m_N, atol=1e-13 * np.abs(Ax).max())


@pytest.mark.parametrize("n", [2, 3, 5])
def test_linear_functions_on_affine_mesh(n):
    pr = Problem(sheared(3), n, 0.0, dirichlet=False, coarse_solver=None, with_schwarz=False)
    a = np.array([0.7, -1.1, 0.4])
    xl = pr.coords @ a
    y = pr.apply_A(xl)
    from oracle.numbering import boundary_mask
    bnd = boundary_mask(pr.l2g, pr.nb_elem, pr.G).astype(bool)
    assert np.max(np.abs(y[~bnd])) < 1e-12 * np.max(np.abs(y))
    # energy of a linear function = |a|^2 * volume
    vol = abs(np.linalg.det(SHEAR))
    assert abs(xl @ y - (a @ a) * vol) < 1e-12


def test_spd_under_dirichlet():
    pr = Problem(lattice_hex_mesh(2, 0.2, 3), 3, 0.0, coarse_solver=None, with_schwarz=False)
    A = pr.assembled().toarray()
    assert np.linalg.eigvalsh(A).min() > 0


def test_spectral_convergence():
    """Error of the discrete solution against u* drops geometrically with n."""
    m = lattice_hex_mesh(2, 0.1, 0)
    errs = []
    for n in range(2, 8):
        pr = Problem(m, n, 1.0, coarse_solver=None, with_schwarz=False)
        A = pr.assembled().tocsc()
        b = pr.load(manufactured_s(pr.coords, 1.0))
        u = spla.spsolve(A, b)
        errs.append(np.max(np.abs(u - manufactured_u(pr.coords))))
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1])
    assert errs[-1] < 1e-4 * errs[0]
