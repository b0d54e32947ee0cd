"""Pins for oracle/schwarz.py (Sec. 4.2, Eq. subd, extended pencil, Eq. z)."""
import numpy as np
import pytest
import scipy.linalg

from synth import lattice_hex_mesh
from oracle.gll import gll_nodes_weights, derivative_matrix
from oracle import schwarz
from oracle.problem import Problem


@pytest.mark.parametrize("n", [2, 3, 5, 7, 8])
def test_pencil_matches_printed_extended_matrix(n):
    t, rho = gll_nodes_weights(n)
    D = derivative_matrix(n)
    d = D.T @ np.diag(rho) @ D
    K, M = schwarz.pencil_matrices(D, rho)
    P = n + 3
    Kp = np.zeros((P, P))
    Kp[1:n + 2, 1:n + 2] = d
    Kp[1, 1] = 2 * d[0, 0]
    Kp[n + 1, n + 1] = 2 * d[n, n]
    Kp[0, 0] = d[1, 1]
    Kp[0, 1] = Kp[1, 0] = d[1, 0]
    Kp[P - 1, P - 1] = d[1, 1]
    Kp[P - 1, P - 2] = Kp[P - 2, P - 1] = d[0, 1]
    np.testing.assert_allclose(K, Kp, atol=1e-12 * n * n)
    Mp = np.diag(np.r_[rho[1], 2 * rho[0], rho[1:n], 2 * rho[n], rho[1]])
    np.testing.assert_allclose(M, Mp, atol=1e-15)
    ev, S = schwarz.pencil_eig(K, M)
    np.testing.assert_allclose(S.T @ M @ S, np.eye(P), atol=1e-12)
    np.testing.assert_allclose(K @ S, M @ S @ np.diag(ev), atol=1e-11 * n * n)
    assert ev.min() > 0


@pytest.mark.parametrize("n,lam", [(2, 0.0), (3, 1.5)])
def test_fast_diagonalisation_equals_dense_solve(n, lam):
    t, rho = gll_nodes_weights(n)
    K, M = schwarz.pencil_matrices(derivative_matrix(n), rho)
    ev, S = schwarz.pencil_eig(K, M)
    rng = np.random.default_rng(3)
    h = rng.uniform(0.05, 0.2, size=(2, 3))
    P = n + 3
    r = rng.standard_normal((2, P, P, P))
    z = schwarz.fast_diag_solve(r, S, ev, h, lam)
    for e in range(2):
        Kb = schwarz.box_matrix(K, M, h[e], lam)
        zd = np.linalg.solve(Kb, 8.0 / np.prod(h[e]) * r[e].ravel())
        np.testing.assert_allclose(z[e].ravel(), zd, rtol=1e-11, atol=1e-11 * np.abs(zd).max())


def _patch_coord_sets(mesh, n):
    pr = Problem(mesh, n, 0.0, coarse_solver=None)
    cent = mesh.xyz[mesh.hex2vert].mean(axis=1)
    order = np.lexsort(np.round(cent, 9).T)
    sets = []
    for e in order:
        ip = pr.ip[e]
        pts = pr.coords[ip[ip >= 0]]
        sets.append(pts[np.lexsort(np.round(pts, 9).T)])
    return sets, pr


def test_patch_nodes_independent_of_orientation_and_numbering():
    a = lattice_hex_mesh(3, 0.2, 11, renumber=False, rotate=False)
    b = lattice_hex_mesh(3, 0.2, 11, renumber=True, rotate=True)
    sa, pa = _patch_coord_sets(a, 3)
    sb, pb = _patch_coord_sets(b, 3)
    for x, y in zip(sa, sb):
        np.testing.assert_allclose(x, y, atol=1e-12)


def test_patch_layer_on_lattice():
    """On an unperturbed, unrotated lattice the i = -1 layer sits at the neighbour's
    first interior GLL line: x = x_face - h (t_1 + 1)/2 ... i.e. one GLL step inside."""
    n, E = 3, 3
    m = lattice_hex_mesh(E, 0.0, 0, renumber=False, rotate=False)
    pr = Problem(m, n, 0.0, coarse_solver=None)
    t = pr.t
    h = 1.0 / E
    step = h * (t[1] - t[0]) / 2
    for e in range(m.n_hex):
        x0 = m.xyz[m.hex2vert[e, 0]]
        for ax in range(3):
            sl = [slice(1, n + 2)] * 3
            sl[ax] = 0
            ids = pr.ip[e][tuple(sl)]
            if x0[ax] == 0.0:
                assert np.all(ids == -1)
            else:
                assert np.all(ids >= 0)
                np.testing.assert_allclose(pr.coords[ids][..., ax], x0[ax] - step, atol=1e-14)
    # edge and corner regions of the box are always absent
    assert np.all(pr.ip[:, 0, 0, :] == -1) and np.all(pr.ip[:, 0, :, 0] == -1)


def test_fine_preconditioner_symmetric_positive():
    pr = Problem(lattice_hex_mesh(2, 0.2, 4), 3, 0.5, coarse_solver=None)
    rng = np.random.default_rng(5)
    free = pr.mask == 0
    x, y = rng.standard_normal(pr.G) * free, rng.standard_normal(pr.G) * free
    Px, Py = pr.apply_Pf(x), pr.apply_Pf(y)
    assert abs(y @ Px - x @ Py) < 1e-12 * abs(y @ Px)
    assert x @ Px > 0


def test_full_box_nodes_extend_the_element_map_on_a_lattice():
    """On an unperturbed (affine) lattice, rotated and renumbered, every filled box node of the
    full patch lies at the element's map evaluated one GLL step beyond the faces."""
    from oracle.problem import Problem
    from oracle.numbering import trilinear_points
    from synth import lattice_hex_mesh
    E, n = 4, 3
    pr = Problem(lattice_hex_mesh(E, 0.0, 7), n, 1.0, coarse_solver=None, patch="full")
    t = pr.t
    ext = np.concatenate([[t[0] - (t[1] - t[0])], t, [t[-1] + (t[-1] - t[-2])]])
    X = trilinear_points(pr.xyz_e, ext)                 # [E, P, P, P, 3]
    present = pr.ip >= 0
    np.testing.assert_allclose(pr.coords[pr.ip[present]], X[present], atol=1e-12)
    # interior elements have every box node; boundary elements miss only the outside layers
    inside = np.all((X > -1e-12) & (X < 1 + 1e-12), axis=-1)
    np.testing.assert_array_equal(present, inside)
    face = Problem(lattice_hex_mesh(E, 0.0, 7), n, 1.0, coarse_solver=None)
    assert (face.ip >= 0).sum() < present.sum()


def test_pencil_variant_without_free_sides_is_the_extended_pencil():
    from oracle import gll
    for n in (2, 5, 8):
        t, rho = gll.gll_nodes_weights(n)
        Dh = gll.derivative_matrix(n)
        K0, M0 = schwarz.pencil_matrices(Dh, rho)
        K1, M1 = schwarz.pencil_variant(Dh, rho, False, False)
        np.testing.assert_array_equal(K1, K0)
        np.testing.assert_array_equal(M1, M0)


@pytest.mark.parametrize("n,lam,seed", [(3, 0.7, 0), (5, 2.0, 3), (7, 0.1, 5)])
def test_insulated_single_box_patch_is_the_exact_element_inverse(n, lam, seed):
    """One undistorted hex with every face insulated: its patch is the element itself with
    free sides on all axes, and the box model is exact, so P^f = A^-1 (any orientation)."""
    from oracle.problem import Problem
    from synth import lattice_hex_mesh
    pr = Problem(lattice_hex_mesh(1, 0.0, seed, box=(0.7, 0.7, 0.7)), n, lam, dirichlet=False,
                 coarse_solver=None, pencils="boundary")
    x = np.random.default_rng(seed).standard_normal(pr.G)
    np.testing.assert_allclose(pr.apply_Pf(pr.apply_A(x)), x, rtol=0, atol=1e-10 * np.abs(x).max())
    ext = Problem(lattice_hex_mesh(1, 0.0, seed, box=(0.7, 0.7, 0.7)), n, lam, dirichlet=False,
                  coarse_solver=None, pencils="extended")
    assert np.abs(ext.apply_Pf(ext.apply_A(x)) - x).max() > 1e-3 * np.abs(x).max()


def test_overlap_weighted_fine_preconditioner():
    """W P^f W with w = cover^-1/2: symmetric positive definite, equal to the plain P^f where
    no patches overlap (one element), and the weights square-sum to one per patch node set."""
    from oracle.problem import Problem
    from synth import lattice_hex_mesh
    pr = Problem(lattice_hex_mesh(3, 0.2, 8), 4, 0.6, coarse_solver=None, weights="cover")
    rng = np.random.default_rng(3)
    free = pr.mask == 0
    x, y = rng.standard_normal(pr.G) * free, rng.standard_normal(pr.G) * free
    assert abs(y @ pr.apply_Pf(x) - x @ pr.apply_Pf(y)) <= 1e-12 * abs(y @ pr.apply_Pf(x))
    assert x @ pr.apply_Pf(x) > 0
    present = pr.ip >= 0
    cover = np.bincount(pr.ip[present], minlength=pr.G)
    np.testing.assert_allclose(cover * pr.w ** 2, 1.0, rtol=1e-14)
    one = Problem(lattice_hex_mesh(1, 0.2, 8), 4, 0.6, coarse_solver=None, weights="cover")
    plain = Problem(lattice_hex_mesh(1, 0.2, 8), 4, 0.6, coarse_solver=None)
    r = rng.standard_normal(one.G)
    np.testing.assert_array_equal(one.apply_Pf(r), plain.apply_Pf(r))
