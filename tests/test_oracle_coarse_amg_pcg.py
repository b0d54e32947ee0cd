"""Pins for oracle/coarse.py (Eq. coarse), oracle/amg.py and oracle/pcg.py (Algorithm 1)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synth import lattice_hex_mesh, manufactured_s, manufactured_u
from oracle import coarse, amg, pcg, gll, geometry, operator
from oracle.problem import Problem


@pytest.fixture(scope="module")
def prob():
    return Problem(lattice_hex_mesh(3, 0.2, 6), 4, 0.8, coarse_solver="exact")


def test_prolongation_is_trilinear_interpolation(prob):
    m = prob.mesh
    for ax in range(3):
        z = coarse.prolong(m.xyz[:, ax], prob.l2g, prob.m_loc, prob.m_N, prob.B, m.hex2vert)
        np.testing.assert_allclose(z, prob.coords[:, ax], atol=1e-14)
    one = coarse.prolong(np.ones(m.n_vert), prob.l2g, prob.m_loc, prob.m_N, prob.B, m.hex2vert)
    np.testing.assert_allclose(one, 1.0, atol=1e-14)


def test_restriction_is_adjoint_of_prolongation(prob):
    m = prob.mesh
    rng = np.random.default_rng(0)
    x, Y = rng.standard_normal(prob.G), rng.standard_normal(m.n_vert)
    R = coarse.restrict(x, prob.l2g, prob.m_loc, prob.m_N, prob.B, m.hex2vert, m.n_vert)
    z = coarse.prolong(Y, prob.l2g, prob.m_loc, prob.m_N, prob.B, m.hex2vert)
    assert abs(R @ Y - x @ z) < 1e-12 * abs(x @ z)


def test_coarse_matrix_is_order_one_operator(prob):
    """A_0 equals the matrix-free operator at n = 1 applied on the vertices."""
    m = prob.mesh
    p1 = Problem(m, 1, prob.lam, dirichlet=False, coarse_solver=None, with_schwarz=False)
    # order-1 nodes are the vertices; map oracle numbering of p1 to vertex ids by position
    vid = np.zeros(p1.G, dtype=np.int64)
    cl2g = coarse.coarse_l2g(m.hex2vert)
    vid[p1.l2g.ravel()] = cl2g.ravel()
    rng = np.random.default_rng(1)
    Zv = rng.standard_normal(m.n_vert)
    y1 = p1.apply_A(Zv[vid])
    fv = prob.free_vert
    A0full = np.zeros(m.n_vert)
    A0full[vid] = y1
    Zf = np.zeros(m.n_vert)
    Zf[fv] = Zv[fv]
    y1f = p1.apply_A(Zf[vid])
    yv = np.zeros(m.n_vert)
    yv[vid] = y1f
    np.testing.assert_allclose(prob.A0 @ Zv[fv], yv[fv], rtol=1e-12, atol=1e-14)


def test_coarse_correction_symmetric_psd(prob):
    rng = np.random.default_rng(2)
    free = prob.mask == 0
    x, y = rng.standard_normal(prob.G) * free, rng.standard_normal(prob.G) * free
    Px, Py = prob.apply_Pc(x), prob.apply_Pc(y)
    assert abs(y @ Px - x @ Py) < 1e-12 * abs(y @ Px)
    assert x @ Px >= 0


def test_pairwise_on_chain():
    n = 9
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    agg, na = amg.pairwise_pass(A)
    assert na == 5
    np.testing.assert_array_equal(agg, [0, 0, 1, 1, 2, 2, 3, 3, 4])


def test_amg_small_is_exact_and_large_is_spd_contraction():
    small = Problem(lattice_hex_mesh(4, 0.2, 1), 2, 1.0, with_schwarz=False)
    H = small.amg
    assert H.sizes() == [small.A0.shape[0]]
    b = np.random.default_rng(3).standard_normal(small.A0.shape[0])
    np.testing.assert_allclose(small.A0 @ H.apply(b), b, atol=1e-12)
    big = Problem(lattice_hex_mesh(16, 0.2, 1), 1, 1.0, with_schwarz=False)
    H = big.amg
    assert len(H.sizes()) >= 2
    A0 = big.A0
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(A0.shape[0]), rng.standard_normal(A0.shape[0])
    assert abs(y @ H.apply(x) - x @ H.apply(y)) < 1e-11 * abs(y @ H.apply(x))
    assert x @ H.apply(x) > 0
    e = x.copy()
    for _ in range(5):
        e2 = e - H.apply(A0 @ e)
        rate = np.sqrt(e2 @ (A0 @ e2) / (e @ (A0 @ e)))
        e = e2
    assert rate < 0.5


def test_cg_on_dense_spd_is_textbook():
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    P = []
    def applyA(p):
        P.append(p.copy())
        return A @ p
    u, it, hist = pcg.pcg(applyA, lambda r: r.copy(), b, rtol=1e-13, maxit=200)
    np.testing.assert_allclose(u, np.linalg.solve(A, b), rtol=1e-10)
    Pm = np.array(P[:10])
    Gm = Pm @ A @ Pm.T
    off = Gm - np.diag(np.diag(Gm))
    assert np.abs(off).max() < 1e-9 * np.abs(np.diag(Gm)).max()
    assert hist[0] == pytest.approx(1.0)


def test_pcg_solution_matches_direct_solve():
    pr = Problem(lattice_hex_mesh(4, 0.1, 0), 3, 0.0)
    b = pr.load(manufactured_s(pr.coords, 0.0))
    u, it, hist = pr.solve(b, rtol=1e-12)
    ud = spla.spsolve(pr.assembled().tocsc(), b)
    assert np.max(np.abs(u - ud)) < 1e-10 * np.max(np.abs(ud))
    r = b - pr.apply_A(u)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11
    assert np.max(np.abs(u - manufactured_u(pr.coords))) < 1e-4


def test_table1_trend_two_scale_flat_fine_only_grows():
    """Table 1 (Sec. 5.1.1): refinement keeps two-scale counts nearly flat while
    fine-only counts grow about twofold per refinement."""
    its = {}
    for E in (4, 8, 16):
        pr = Problem(lattice_hex_mesh(E, 0.1, 0), 3, 0.0)
        b = pr.load(np.ones(pr.G))
        its[E] = (pr.solve(b, precond="two-scale")[1], pr.solve(b, precond="fine")[1])
    two = [its[E][0] for E in (4, 8, 16)]
    fine = [its[E][1] for E in (4, 8, 16)]
    assert two[2] <= 1.5 * two[1]
    assert fine[2] >= 1.6 * fine[1]
    assert fine[2] > 1.5 * two[2]


def _q1_free(E, seed=1, lam=1.0):
    return Problem(lattice_hex_mesh(E, 0.2, seed), 1, lam, with_schwarz=False, coarse_solver="kcycle")


def test_unsmoothed_aggregation_is_piecewise_constant_galerkin():
    pr = _q1_free(28)
    H = pr.amg
    assert len(H.levels) >= 2
    A = pr.A0
    for Al, Dinv, P in H.levels:
        P = sp.csr_matrix(P)
        assert np.all(np.diff(P.indptr) == 1) and np.all(P.data == 1.0)   # one aggregate per unknown
        assert max(np.bincount(P.indices)) <= 4                           # two pairwise passes
        Ac = P.T @ Al @ P
        one, onec = np.ones(Al.shape[0]), np.ones(P.shape[1])
        assert abs(onec @ (Ac @ onec) - one @ (Al @ one)) <= 1e-12 * abs(one @ (Al @ one))


def test_kcycle_on_two_levels_is_the_two_grid_cycle():
    pr = _q1_free(14)
    H = pr.amg
    assert len(H.levels) == 1
    A, Dinv, P = H.levels[0]
    Ad = A.toarray()
    Pd = P.toarray()
    Ac = Pd.T @ Ad @ Pd
    b = np.random.default_rng(7).standard_normal(A.shape[0])
    x = (2.0 / 3.0) * Dinv * b
    x = x + Pd @ np.linalg.solve(Ac, Pd.T @ (b - Ad @ x))
    x = x + (2.0 / 3.0) * Dinv * (b - Ad @ x)
    np.testing.assert_allclose(H.kcycle(b), x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_kcycle_inner_correction_is_galerkin_on_two_directions():
    pr = _q1_free(24)
    H = pr.amg
    assert len(H.levels) >= 2
    A1 = H.levels[1][0]
    rc = np.random.default_rng(8).standard_normal(A1.shape[0])
    ec, c1, c2 = H.coarse_correction(rc, 1)
    res = rc - A1 @ ec
    for c in (c1, c2):
        assert abs(c @ res) <= 1e-10 * np.linalg.norm(c) * np.linalg.norm(rc)


def test_flexible_cg_with_kcycle_is_h_independent():
    its = []
    for E in (18, 24, 32):          # one, two and three aggregation levels above the dense one
        pr = _q1_free(E)
        b = np.random.default_rng(9).standard_normal(pr.A0.shape[0])
        its.append(pcg.fpcg(lambda v: pr.A0 @ v, pr.amg.apply, b, rtol=1e-8)[1])
    assert max(its) - min(its) <= 3 and max(its) <= 20, its


def test_fpcg_with_fixed_spd_preconditioner_is_pcg():
    pr = Problem(lattice_hex_mesh(3, 0.2, 4), 3, 1.0, coarse_solver="exact")
    b = pr.load(np.random.default_rng(10).standard_normal(pr.G))
    h0 = pcg.pcg(pr.apply_A, pr.apply_P, b, 1e-10)[2]
    h1 = pcg.fpcg(pr.apply_A, pr.apply_P, b, 1e-10)[2]
    assert len(h0) == len(h1)
    np.testing.assert_allclose(h1, h0, rtol=1e-6, atol=1e-13)
