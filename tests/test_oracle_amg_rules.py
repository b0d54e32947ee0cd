"""Pins of the oracle's aggregation rule (oracle/amg.py) on cases small enough to work out by
hand from the rule as written (the paper, Sec. 4.1.1, names aggregation AMG but does not fix
the aggregation; the library implements the same written rule independently). Each expected
value below was derived by stepping through the rule by hand, not by running the oracle:
a mistake in the visiting order, the strength threshold, the sign test, the tie rule, the
number of passes, the Galerkin recomposition or the smoothing weight fails one of them."""
import numpy as np
import scipy.sparse as sp

from oracle import amg


def _grid_laplacian(nx, ny):
    """5-point Laplacian on an nx x ny grid, row-major numbering (node x + nx y)."""
    n = nx * ny
    rows, cols, vals = [], [], []
    for y in range(ny):
        for x in range(nx):
            i = x + nx * y
            rows.append(i); cols.append(i); vals.append(4.0)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < nx and 0 <= y + dy < ny:
                    rows.append(i); cols.append(x + dx + nx * (y + dy)); vals.append(-1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def test_pairwise_on_3x3_grid():
    """Equal strengths everywhere: visiting 0..8, each free node pairs with its lowest-numbered
    free neighbour. 0 takes 1 (not 3: the tie keeps the lower j); 2 takes 5 (1 is taken);
    3 takes 4; 6 takes 7 (3 is taken); 8 has no free neighbour left and stays alone."""
    agg, na = amg.pairwise_pass(_grid_laplacian(3, 3))
    assert na == 5
    np.testing.assert_array_equal(agg, [0, 0, 1, 2, 2, 1, 3, 3, 4])


def test_weak_neighbour_is_not_taken():
    """Node 2's strongest connection (to 1, s = 1) is already aggregated; its only free
    neighbour 3 has s = 0.2 < 0.25 x 1, below the strength threshold, so 2 stays alone, and
    so does 3 (its only neighbour is taken)."""
    A = sp.csr_matrix(np.array([[4.0, -1.0, 0.0, 0.0],
                                [-1.0, 4.0, -1.0, 0.0],
                                [0.0, -1.0, 4.0, -0.2],
                                [0.0, 0.0, -0.2, 4.0]]))
    agg, na = amg.pairwise_pass(A)
    assert na == 3
    np.testing.assert_array_equal(agg, [0, 0, 1, 2])


def test_strong_enough_neighbour_is_taken():
    """The same with s_23 = 0.3 >= 0.25: now 2 and 3 pair."""
    A = sp.csr_matrix(np.array([[4.0, -1.0, 0.0, 0.0],
                                [-1.0, 4.0, -1.0, 0.0],
                                [0.0, -1.0, 4.0, -0.3],
                                [0.0, 0.0, -0.3, 4.0]]))
    agg, na = amg.pairwise_pass(A)
    assert na == 2
    np.testing.assert_array_equal(agg, [0, 0, 1, 1])


def test_positive_couplings_are_ignored():
    """A positive off-diagonal entry is no connection: node 0's only negative neighbour is 2,
    although a_01 = +1.5 is the largest in magnitude; then 1 pairs with 3."""
    A = sp.csr_matrix(np.array([[4.0, 1.5, -1.0, 0.0],
                                [1.5, 4.0, 0.0, -1.0],
                                [-1.0, 0.0, 4.0, 0.0],
                                [0.0, -1.0, 0.0, 4.0]]))
    agg, na = amg.pairwise_pass(A)
    assert na == 2
    np.testing.assert_array_equal(agg, [0, 1, 0, 1])


def test_near_ties_keep_the_lower_index():
    """A later neighbour replaces the current choice only when stronger by more than a factor
    1 + 1e-10: s = 1 + 1e-12 keeps neighbour 1, s = 1.001 takes neighbour 2."""
    for s2, expect in ((1.0 + 1e-12, [0, 0, 1]), (1.001, [0, 1, 0])):
        A = sp.csr_matrix(np.array([[4.0, -1.0, -s2],
                                    [-1.0, 4.0, 0.0],
                                    [-s2, 0.0, 4.0]]))
        agg, na = amg.pairwise_pass(A)
        assert na == 2
        np.testing.assert_array_equal(agg, expect)


def test_three_passes_on_a_chain_give_aggregates_of_eight_and_the_smoothed_prolongator():
    """On the 1D chain (2, -1) with 3,000 unknowns: a pairwise pass pairs (0,1), (2,3), ...;
    the Galerkin product of a chain with such pairs is again the chain (2, -1) (row sums of the
    2x2 blocks), so the second and third passes pair again: the tentative aggregates are the
    runs of 8 consecutive unknowns, 375 of them (375 <= 2,048 ends the hierarchy there).
    The smoothing weight is (4/3) / max_i sum_j |a_ij| / a_ii = (4/3) / 2 = 2/3, so
    P = T - (2/3) D^-1 A T with D = 2 I: inside a run (A T) = -1 + 2 - 1 = 0 and P = 1; at a
    run's end next to another run (A T) = 2 - 1 = 1 in its own column and -1 in the neighbour's,
    so P = 1 - 1/3 = 2/3 and 1/3; at the chain's two ends the row sum of A is 1 (the truncated
    chain), so P = 2/3 there too, with no neighbouring column."""
    n = 3000
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    H = amg.AMG(A)
    assert H.sizes() == [3000, 375]
    P = H.levels[0][2].toarray()
    assert P.shape == (3000, 375)
    expect = np.zeros((n, n // 8))
    for i in range(n):
        a = i // 8
        first, last = i % 8 == 0, i % 8 == 7
        expect[i, a] = 2.0 / 3.0 if (first or last) else 1.0
        if first and a > 0:
            expect[i, a - 1] = 1.0 / 3.0
        if last and a < n // 8 - 1:
            expect[i, a + 1] = 1.0 / 3.0
    np.testing.assert_allclose(P, expect, rtol=0, atol=1e-15)
    # the coarse operator is the Galerkin product, and the dense coarsest solve inverts it
    Ac = (sp.csr_matrix(P).T @ A @ sp.csr_matrix(P)).toarray()
    np.testing.assert_allclose(H.coarsest_inv @ Ac, np.eye(375), atol=1e-9)


def test_kcycle_hierarchy_is_unsmoothed_pairs_of_pairs():
    """The paper's cycle (kind "kcycle") takes two pairwise passes and no smoothing: on the
    chain the aggregates are runs of 4 and the prolongator is their 0/1 indicator."""
    n = 4096
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    H = amg.AMG(A, kind="kcycle")
    assert H.sizes() == [4096, 1024]
    P = H.levels[0][2].toarray()
    expect = np.zeros((n, n // 4))
    expect[np.arange(n), np.arange(n) // 4] = 1.0
    np.testing.assert_array_equal(P, expect)


def test_coarsening_that_stalls_ends_in_the_dense_solve():
    """With no negative coupling every unknown stays a singleton, so a level would keep all
    3,000 unknowns (more than 3/4): the hierarchy stops at once and the dense solve takes the
    whole matrix."""
    n = 3000
    d = np.linspace(1.0, 2.0, n)
    H = amg.AMG(sp.diags(d).tocsr())
    assert H.sizes() == [3000]
    np.testing.assert_allclose(np.diag(H.coarsest_inv), 1.0 / d, rtol=1e-14)
