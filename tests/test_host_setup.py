"""The library's host set-up (C++, no CUDA) against the oracle, on the CPU.

Tables are compared by node position, since the library and the oracle number
nodes differently (any bijection is allowed).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import lattice_hex_mesh
from oracle.problem import Problem
from oracle import schwarz
from host_harness import load, HostTables


@pytest.fixture(scope="module")
def lib():
    return load()


def match(ref_xyz, lib_xyz):
    """perm with lib_xyz[perm] == ref_xyz."""
    oi = np.lexsort(np.round(ref_xyz, 9).T)
    gi = np.lexsort(np.round(lib_xyz, 9).T)
    perm = np.empty_like(gi)
    perm[oi] = gi
    assert np.abs(lib_xyz[perm] - ref_xyz).max() < 1e-12
    return perm


@pytest.mark.parametrize("E,n,a,seed,patch", [(1, 3, 0.1, 0, "face"), (3, 3, 0.2, 1, "face"), (2, 5, 0.15, 2, "face"),
                                              (4, 2, 0.2, 3, "face"), (2, 2, 0.1, 4, "face"), (3, 8, 0.2, 5, "face"),
                                              (3, 3, 0.2, 1, "full"), (4, 2, 0.2, 3, "full"), (3, 5, 0.1, 6, "full")])
def test_numbering_patch_and_tables(lib, E, n, a, seed, patch):
    mesh = lattice_hex_mesh(E, a, seed)
    H = HostTables(lib, mesh, n, 0.3, patch=patch)
    assert H.rc == 0
    ref = Problem(mesh, n, 0.3, coarse_solver=None, patch=patch)
    assert H.G == ref.G
    perm = match(ref.coords, H.coords)          # oracle dof -> lib dof
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))            # lib dof -> oracle dof
    np.testing.assert_array_equal(H.boundary[perm], ref.mask)
    p, P = n + 1, n + 3
    # l2g: library element e is input element elem_perm[e]; local order i fastest
    l2g = H.l2g.reshape(H.ne, p, p, p)          # [e, k, j, i]
    ref_l2g = ref.l2g[H.elem_perm].transpose(0, 3, 2, 1)
    np.testing.assert_array_equal(inv[l2g], ref_l2g)
    # element-interior nodes come first: DOF e m^3 + a + m (b + m c) at local (a+1, b+1, c+1)
    m = n - 1
    interior = l2g[:, 1:n, 1:n, 1:n]             # [e, c, b, a]
    np.testing.assert_array_equal(interior.reshape(-1), np.arange(H.ne * m ** 3))
    shared = np.ones((p, p, p), dtype=bool)
    shared[1:n, 1:n, 1:n] = False
    assert l2g[:, shared].min() == H.ne * m ** 3 and l2g[:, shared].max() == H.G - 1
    # patch tables
    ip = H.ip.reshape(H.ne, P, P, P)
    ref_ip = ref.ip[H.elem_perm].transpose(0, 3, 2, 1)
    lib_ip_in_ref = np.where(ip >= 0, inv[np.maximum(ip, 0)], -1)
    np.testing.assert_array_equal(lib_ip_in_ref, ref_ip)
    # box sizes, GLL, D
    np.testing.assert_allclose(H.hbox.reshape(-1, 3), ref.h[H.elem_perm], rtol=1e-14)
    np.testing.assert_allclose(H.t, ref.t, atol=1e-15)
    np.testing.assert_allclose(H.rho, ref.rho, rtol=1e-14)
    np.testing.assert_allclose(H.D.reshape(p, p), ref.Dh, atol=1e-12 * n * n)
    # pencil: compare the operator S diag(1/(ev+1)) S^T (eigenvector sign/order free)
    S = H.S.reshape(P, P)
    Bl = S @ np.diag(1.0 / (H.ev + 1.0)) @ S.T
    Br = ref.S @ np.diag(1.0 / (ref.ev + 1.0)) @ ref.S.T
    np.testing.assert_allclose(Bl, Br, atol=1e-12 * np.abs(Br).max())
    np.testing.assert_allclose(np.sort(H.ev), np.sort(ref.ev), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("E,n,lam,kind", [(16, 1, 1.0, 0), (20, 2, 0.0, 0), (24, 1, 0.5, 1), (20, 2, 0.0, 1)])
def test_amg_hierarchy_matches_oracle(lib, E, n, lam, kind):
    mesh = lattice_hex_mesh(E, 0.2, 1)
    H = HostTables(lib, mesh, n, lam, amg_kind=kind)
    assert H.rc == 0
    ref = Problem(mesh, n, lam, with_schwarz=False, coarse_solver=("amg", "kcycle")[kind])
    np.testing.assert_array_equal(H.keep, ref.free_vert)
    assert H.amg_sizes == ref.amg.sizes()
    for l, (A, Dinv, Pm) in enumerate(ref.amg.levels):
        for which, M in ((0, A), (1, Pm)):
            ptr, col, val = H.amg_level(l, which)
            Ml = sp.csr_matrix((val, col, ptr), shape=M.shape)
            diff = abs(Ml - M).max()
            assert diff <= 1e-12 * abs(M).max(), (l, which, diff)
    ci = H.coarsest_inv()
    np.testing.assert_allclose(ci, ref.amg.coarsest_inv, atol=1e-10 * np.abs(ref.amg.coarsest_inv).max())


def test_nonmanifold_mesh_rejected(lib):
    mesh = lattice_hex_mesh(2, 0.0, 0)
    bad = mesh.hex2vert.copy()
    # a third hex on an existing face
    extra = bad[0].copy()
    mesh.hex2vert = np.vstack([bad, extra[None, :]])
    H = HostTables(lib, mesh, 2, 0.0)
    assert H.rc == -1


@pytest.mark.parametrize("N,layers,n,seed", [(2, 2, 3, 1), (3, 1, 4, 2), (2, 3, 2, 3)])
def test_tables_on_irregular_valence_meshes(lib, N, layers, n, seed):
    """Numbering, patch tables, box sizes and the AMG hierarchy on an all-hex mesh whose
    edges have valence 1 to 8 (triangles split into quads, extruded)."""
    from synth import split_triangle_hex_mesh
    mesh = split_triangle_hex_mesh(N, layers, a=0.1, seed=seed)
    H = HostTables(lib, mesh, n, 0.4)
    assert H.rc == 0
    ref = Problem(mesh, n, 0.4, with_schwarz=True)
    assert H.G == ref.G
    perm = match(ref.coords, H.coords)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    np.testing.assert_array_equal(H.boundary[perm], ref.mask)
    p, P = n + 1, n + 3
    l2g = H.l2g.reshape(H.ne, p, p, p)
    np.testing.assert_array_equal(inv[l2g], ref.l2g[H.elem_perm].transpose(0, 3, 2, 1))
    ip = H.ip.reshape(H.ne, P, P, P)
    lib_ip_in_ref = np.where(ip >= 0, inv[np.maximum(ip, 0)], -1)
    np.testing.assert_array_equal(lib_ip_in_ref, ref.ip[H.elem_perm].transpose(0, 3, 2, 1))
    np.testing.assert_allclose(H.hbox.reshape(-1, 3), ref.h[H.elem_perm], rtol=1e-14)


@pytest.mark.parametrize("E,n,lam", [(20, 2, 0.0), (32, 1, 0.7)])
def test_fused_vcycle_matrices_reproduce_the_cycle(lib, E, n, lam):
    """Per level, the two sparse products the GPU runs (b_c = M b, x = N b + Q x_c) equal the
    V(1,1) cycle's steps done one by one with Jacobi weight 2/3: pre-smoothing from zero,
    residual, restriction by P^T; prolongation and post-smoothing."""
    mesh = lattice_hex_mesh(E, 0.2, 1)
    H = HostTables(lib, mesh, n, lam, amg_kind=0)
    assert H.rc == 0 and len(H.amg_sizes) >= 2
    rng = np.random.default_rng(E + n)
    w = 2.0 / 3.0
    for l in range(len(H.amg_sizes) - 1):
        A, P, M, N, Q = (H.amg_matrix(l, k) for k in range(5))
        dinv = 1.0 / A.diagonal()
        b = rng.standard_normal(A.shape[0])
        xc = rng.standard_normal(P.shape[1])
        x = w * dinv * b
        bc = P.T @ (b - A @ x)
        x1 = x + P @ xc
        out = x1 + w * dinv * (b - A @ x1)
        np.testing.assert_allclose(M @ b, bc, rtol=0, atol=1e-13 * np.abs(bc).max())
        np.testing.assert_allclose(N @ b + Q @ xc, out, rtol=0, atol=1e-13 * np.abs(out).max())
