"""Pins for the synthetic meshes, oracle/numbering.py and oracle/geometry.py."""
import numpy as np
import pytest

from synth import lattice_hex_mesh, VTK_CORNER_BITS
from oracle.gll import gll_nodes_weights
from oracle import numbering, geometry


def test_mesh_generator_stays_in_unit_cube_and_positive():
    m = lattice_hex_mesh(6, 0.2, 3)
    assert m.xyz.min() == 0.0 and m.xyz.max() == 1.0
    t, rho = gll_nodes_weights(4)
    _, _, detJ = geometry.geometric_factors(m.xyz[m.hex2vert], t, rho)
    assert detJ.min() > 0


@pytest.mark.parametrize("E,n", [(1, 3), (2, 4), (3, 2)])
def test_global_count_and_multiplicity(E, n):
    m = lattice_hex_mesh(E, 0.15, 1)
    t, _ = gll_nodes_weights(n)
    l2g, X = numbering.local_to_global(m, t)
    assert X.shape[0] == (E * n + 1) ** 3
    mult = np.bincount(l2g.ravel())
    # corner of the cube: 1 copy; interior lattice vertex: 8 copies
    assert mult.min() == 1 and mult.max() == (8 if E > 1 else 1)
    assert np.sum(mult) == m.n_hex * (n + 1) ** 3


def test_scatter_gather_adjoint():
    m = lattice_hex_mesh(3, 0.2, 2)
    t, _ = gll_nodes_weights(3)
    l2g, X = numbering.local_to_global(m, t)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(X.shape[0])
    rl = rng.standard_normal(l2g.shape)
    lhs = numbering.gather(rl, l2g, X.shape[0]) @ x
    rhs = np.sum(rl * numbering.scatter(x, l2g))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_boundary_mask_is_cube_surface():
    m = lattice_hex_mesh(4, 0.2, 5)
    t, _ = gll_nodes_weights(3)
    l2g, X = numbering.local_to_global(m, t)
    nb, _ = numbering.face_neighbours(m)
    mask = numbering.boundary_mask(l2g, nb, X.shape[0])
    on = ((np.abs(X) < 1e-13) | (np.abs(X - 1) < 1e-13)).any(axis=1)
    assert np.array_equal(on, mask.astype(bool))


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_mass_sums_to_volume(n):
    m = lattice_hex_mesh(3, 0.2, 4)
    t, rho = gll_nodes_weights(n)
    _, mloc, _ = geometry.geometric_factors(m.xyz[m.hex2vert], t, rho)
    assert abs(mloc.sum() - 1.0) < 1e-13
    # per-element volume from an independent 2x2x2 Gauss rule on the trilinear map
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    J = geometry.jacobians(m.xyz[m.hex2vert], g)
    vol = np.linalg.det(J).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(mloc.sum(axis=(1, 2, 3)), vol, rtol=1e-13)


def test_box_sizes_on_lattice():
    m = lattice_hex_mesh(5, 0.0, 0)
    h = geometry.element_box_sizes(m.xyz[m.hex2vert])
    np.testing.assert_allclose(h, 0.2, rtol=1e-14)
