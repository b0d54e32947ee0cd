"""GPU path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerance: 1e-12 relative (max-norm) for the operator and the preconditioner
in FP64; PCG is compared at equal iteration counts with the histories within
1e-10 and the solutions within 1e-10 (rounding-order differences grow slowly
through the recurrences).
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s, manufactured_u

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


def _pair(*a, **k):
    from gpu_util import Pair
    return Pair(*a, **k)


CASES = [  # E, n, lam, a, seed
    (1, 3, 0.0, 0.1, 0), (2, 4, 1.3, 0.2, 1), (4, 3, 0.0, 0.1, 0), (3, 2, 0.5, 0.2, 2),
    (2, 5, 2.0, 0.2, 3), (2, 6, 0.0, 0.15, 4), (2, 7, 1.0, 0.2, 5), (2, 8, 0.7, 0.2, 6),
]


@pytest.mark.parametrize("E,n,lam,a,seed", CASES)
@pytest.mark.parametrize("geom", ["stored", "recompute"])
def test_operator_parity(E, n, lam, a, seed, geom):
    from gpu_util import rel_err
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, geom=geom, coarse=False, schwarz=False)
    x = np.random.default_rng(seed).standard_normal(P.ref.G)
    y = P.to_ref(P.gpu.apply_A(P.to_gpu(x)))
    assert rel_err(y, P.ref.apply_A(x)) <= TOL
    np.testing.assert_array_equal(P.to_ref(P.gpu.mask()), P.ref.mask)
    assert rel_err(P.to_ref(P.gpu.mass()), P.ref.m_N) <= TOL


def test_operator_neumann_nullspace():
    from gpu_util import rel_err
    for lam in (0.0, 1.5):
        P = _pair(lattice_hex_mesh(3, 0.2, 7), 4, lam, neumann=True, coarse=False, schwarz=False)
        one = torch.ones(P.gpu.n_dof, dtype=torch.float64, device="cuda")
        y = P.to_ref(P.gpu.apply_A(one))
        np.testing.assert_allclose(y, lam * P.ref.m_N, atol=1e-13 * np.abs(P.ref.m_N).max() * max(lam, 1.0) * 50)
        x = np.random.default_rng(1).standard_normal(P.ref.G)
        assert rel_err(P.to_ref(P.gpu.apply_A(P.to_gpu(x))), P.ref.apply_A(x)) <= TOL


@pytest.mark.parametrize("E,n,lam,a,seed", [(2, 3, 0.0, 0.1, 0), (4, 3, 0.0, 0.1, 0), (3, 5, 1.0, 0.2, 1),
                                            (2, 8, 0.5, 0.2, 2), (10, 2, 1.0, 0.2, 3)])
def test_preconditioner_parity(E, n, lam, a, seed):
    from gpu_util import rel_err
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam)
    r = np.random.default_rng(seed + 10).standard_normal(P.ref.G)
    rg = P.to_gpu(r)
    assert rel_err(P.to_ref(P.gpu.apply_P(rg, "fine")), P.ref.apply_Pf(r)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(rg, "coarse")), P.ref.apply_Pc(r)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(rg, "two-scale")), P.ref.apply_P(r)) <= TOL


@pytest.mark.parametrize("E,n,lam,a,seed,pc", [(4, 3, 0.0, 0.1, 0, "two-scale"), (3, 4, 1.0, 0.2, 1, "fine"),
                                               (10, 2, 1.0, 0.2, 3, "two-scale"), (3, 3, 0.5, 0.2, 2, "none")])
def test_pcg_parity(E, n, lam, a, seed, pc):
    from gpu_util import hist_atol
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam)
    b = P.ref.load(manufactured_s(P.ref.coords, lam))
    u, it_ref, hist_ref = P.ref.solve(b, rtol=1e-8, maxit=500, precond=pc)
    for prec in ("fp64", "fp64_native"):     # double-FP32 element kernels (default) and binary64
        P.gpu.set_precision(prec)
        x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8, maxit=500, precond=pc)
        assert rc == 0
        assert it == it_ref
        np.testing.assert_allclose(hist, hist_ref, rtol=1e-9, atol=hist_atol(1e-14, prec))
        ug = P.to_ref(x)
        assert np.max(np.abs(ug - u)) <= 1e-10 * np.max(np.abs(u))
        assert tr <= 2e-8
        # the discrete solution approximates the manufactured one
        assert np.max(np.abs(ug - manufactured_u(P.ref.coords))) < 0.05


def test_pcg_config1_golden():
    """4^3 hexes, +-10 %, seed 0, n = 3, lambda = 0: iteration count and history of the
    committed oracle golden file."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config1_oracle.json")))
    from gpu_util import hist_atol
    P = _pair(lattice_hex_mesh(4, 0.1, 0), 3, 0.0)
    b = P.ref.load(manufactured_s(P.ref.coords, 0.0))
    for prec in ("fp64", "fp64_native"):
        P.gpu.set_precision(prec)
        x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
        assert it == gold["iterations"]
        np.testing.assert_allclose(hist, gold["residual_history"], rtol=1e-9, atol=hist_atol(1e-14, prec))


def test_solve_is_deterministic():
    P = _pair(lattice_hex_mesh(6, 0.2, 4), 4, 1.0)
    b = P.to_gpu(P.ref.load(manufactured_s(P.ref.coords, 1.0)))
    x1, _, it1, h1, _ = P.gpu.solve(b)
    x2, _, it2, h2, _ = P.gpu.solve(b)
    assert it1 == it2 and np.array_equal(h1, h2)
    assert torch.equal(x1, x2)


def test_edge_cases():
    from gpu_util import rel_err
    # single element, all boundary: only interior nodes free, no free vertex (no coarse space)
    P = _pair(lattice_hex_mesh(1, 0.1, 0), 2, 0.0)
    b = P.ref.load(np.ones(P.ref.G))
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b))
    u, it_ref, _ = P.ref.solve(b)
    assert rc == 0 and it == it_ref and rel_err(P.to_ref(x), u) < 1e-10
    # zero right-hand side: zero iterations, zero solution
    x, rc, it, hist, tr = P.gpu.solve(torch.zeros(P.gpu.n_dof, dtype=torch.float64, device="cuda"))
    assert rc == 0 and it == 0 and float(x.abs().max()) == 0.0
    # maxit reached
    P = _pair(lattice_hex_mesh(3, 0.2, 1), 3, 0.0)
    b = P.to_gpu(P.ref.load(np.ones(P.ref.G)))
    x, rc, it, hist, tr = P.gpu.solve(b, maxit=3)
    assert rc == 1 and it == 3 and len(hist) == 4
    # NaN in the load is reported, not propagated silently
    bn = b.clone()
    bn[int(torch.nonzero(P.gpu.mask() == 0)[0])] = float("nan")
    from paper_1506_05996_gb300.sem import SemError
    with pytest.raises(SemError):
        P.gpu.solve(bn)
    # a mirrored hex (negative Jacobian) is refused
    from synth import lattice_hex_mesh as lhm
    m = lhm(2, 0.0, 0)
    m.hex2vert[0] = m.hex2vert[0][[1, 0, 3, 2, 5, 4, 7, 6]]
    from paper_1506_05996_gb300.sem import SemProblem
    with pytest.raises(SemError) as ei:
        SemProblem(m.xyz, m.hex2vert, 3, 0.0)
    assert ei.value.code == -2


def test_operator_parity_at_full_size():
    """32^3 hexes, +-20 % (seed 1), n = 7, lambda = 1 (about 11.4 M DOFs): every DOF of
    A x against the oracle's matrix-free apply, stored and recomputed geometry."""
    from gpu_util import rel_err, Pair
    from paper_1506_05996_gb300.sem import SemProblem
    mesh = lattice_hex_mesh(32, 0.2, 1)
    P = _pair(mesh, 7, 1.0, geom="stored", coarse=False, schwarz=False)
    x = np.random.default_rng(2).standard_normal(P.ref.G)
    y_ref = P.ref.apply_A(x)
    assert rel_err(P.to_ref(P.gpu.apply_A(P.to_gpu(x))), y_ref) <= TOL
    xg = P.to_gpu(x)
    coords = P.gpu.dof_coords().clone()
    P.gpu.close()
    rec = SemProblem(mesh.xyz, mesh.hex2vert, 7, 1.0, geom="recompute")
    assert torch.equal(rec.dof_coords(), coords)      # same numbering in both variants
    y = rec.apply_A(xg).cpu().numpy()[P.perm]
    assert rel_err(y, y_ref) <= TOL


@pytest.mark.parametrize("E,n,lam,seed", [(3, 3, 0.5, 21), (2, 6, 1.0, 22)])
def test_full_patch_parity(E, n, lam, seed):
    """P^f with the edge and corner layers filled (SEM_PATCH_FULL) against the oracle."""
    from gpu_util import rel_err
    from oracle.problem import Problem
    from paper_1506_05996_gb300.sem import SemProblem
    mesh = lattice_hex_mesh(E, 0.2, seed)
    gpu = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, patch="full")
    ref = Problem(mesh, n, lam, patch="full")
    X = gpu.dof_coords().cpu().numpy()
    oi, gi = np.lexsort(np.round(ref.coords, 9).T), np.lexsort(np.round(X, 9).T)
    perm = np.empty_like(gi)
    perm[oi] = gi
    r = np.random.default_rng(seed).standard_normal(ref.G) * (ref.mask == 0)
    rg = torch.zeros(gpu.n_dof, dtype=torch.float64, device="cuda")
    rg[torch.as_tensor(perm, device="cuda")] = torch.as_tensor(r, device="cuda")
    assert rel_err(gpu.apply_P(rg, "fine").cpu().numpy()[perm], ref.apply_Pf(r)) <= TOL
    b = ref.load(manufactured_s(ref.coords, lam))
    bg = torch.zeros_like(rg)
    bg[torch.as_tensor(perm, device="cuda")] = torch.as_tensor(b, device="cuda")
    assert gpu.solve(bg)[2] == ref.solve(b)[1]
    gpu.close()


@pytest.mark.parametrize("E,n,lam,seed", [(3, 4, 0.6, 23), (2, 6, 2.0, 24), (2, 3, 0.0, 25)])
def test_neumann_patch_parity(E, n, lam, seed):
    """P^f with natural-boundary pencils on insulated faces (Neumann) against the oracle;
    lam = 0 too: P^f alone stays defined (the box problems are not singular)."""
    from gpu_util import rel_err
    P = _pair(lattice_hex_mesh(E, 0.2, seed), n, lam, neumann=True, coarse=False)
    r = np.random.default_rng(seed).standard_normal(P.ref.G)
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), P.ref.apply_Pf(r)) <= TOL


def test_partial_dirichlet_mask_patch_parity():
    """Dirichlet on the x = 0 face only (sem_set_mask): the other boundary faces take the
    natural-boundary pencil, in the library and the oracle alike."""
    from gpu_util import rel_err
    from oracle.problem import Problem
    mesh = lattice_hex_mesh(3, 0.2, 26)
    P = _pair(mesh, 4, 0.8, neumann=True, coarse=False)
    mask = (np.abs(P.ref.coords[:, 0]) < 1e-12).astype(np.uint8)
    mg = torch.zeros(P.gpu.n_dof, dtype=torch.uint8, device="cuda")
    mg[torch.as_tensor(P.perm, device="cuda")] = torch.as_tensor(mask, device="cuda")
    from paper_1506_05996_gb300 import sem
    sem.sem_set_mask(P.gpu.h, mg)
    ref = Problem(mesh, 4, 0.8, dirichlet=False, coarse_solver=None)
    ref.mask = mask
    ref._setup_schwarz()
    r = np.random.default_rng(27).standard_normal(ref.G)
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), ref.apply_Pf(r)) <= TOL


@pytest.mark.parametrize("n,lam", [(3, 0.7), (7, 0.1)])
def test_insulated_single_box_patch_is_exact_inverse(n, lam):
    """One undistorted hex, every face insulated: P^f A x = x (the box model is exact)."""
    from paper_1506_05996_gb300.sem import SemProblem
    mesh = lattice_hex_mesh(1, 0.0, 3, box=(0.7, 0.7, 0.7))
    pr = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, neumann=True)
    x = torch.randn(pr.n_dof, dtype=torch.float64, device="cuda")
    y = pr.apply_P(pr.apply_A(x), "fine")
    assert float((y - x).abs().max()) <= 1e-10 * float(x.abs().max())
    pr.close()


@pytest.mark.parametrize("E,n,lam,seed", [(3, 4, 0.6, 28), (2, 7, 1.0, 29)])
def test_overlap_weighted_patch_parity(E, n, lam, seed):
    """W P^f W (sem_set_weights) against the oracle, P^f and the whole solve."""
    from gpu_util import rel_err
    from oracle.problem import Problem
    from paper_1506_05996_gb300 import sem
    mesh = lattice_hex_mesh(E, 0.2, seed)
    P = _pair(mesh, n, lam)
    ref = Problem(mesh, n, lam, weights="cover")
    sem.sem_set_weights(P.gpu.h, 1)
    r = np.random.default_rng(seed).standard_normal(ref.G)
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), ref.apply_Pf(r)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r))), ref.apply_P(r)) <= TOL
    b = ref.load(manufactured_s(ref.coords, lam))
    _, it_ref, h_ref = ref.solve(b)
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b))
    assert rc == 0 and it == it_ref and tr <= 1e-8
    from gpu_util import hist_atol
    np.testing.assert_allclose(hist, h_ref, rtol=1e-9, atol=hist_atol(1e-15))
    sem.sem_set_weights(P.gpu.h, 0)
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), P.ref.apply_Pf(r)) <= TOL


@pytest.mark.parametrize("N,layers,n,lam,seed", [(3, 2, 3, 0.5, 1), (2, 2, 6, 1.0, 2)])
def test_irregular_valence_mesh_parity(N, layers, n, lam, seed):
    """Operator, preconditioner and solve on an all-hex mesh with edge valences 1 to 8."""
    from gpu_util import Pair, rel_err
    from synth import split_triangle_hex_mesh
    mesh = split_triangle_hex_mesh(N, layers, a=0.1, seed=seed)
    for geom in ("stored", "recompute"):
        P = Pair(mesh, n, lam, geom=geom)
        x = np.random.default_rng(seed).standard_normal(P.ref.G)
        assert rel_err(P.to_ref(P.gpu.apply_A(P.to_gpu(x))), P.ref.apply_A(x)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(x), "fine")), P.ref.apply_Pf(x)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(x), "coarse")), P.ref.apply_Pc(x)) <= TOL
    b = P.ref.load(np.ones(P.ref.G))
    u_ref, it_ref, h_ref = P.ref.solve(b)
    xs, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b))
    # these meshes are poorly conditioned (tens of iterations): rounding-order differences
    # grow along the CG trajectory, so the early history, the count and the solution are
    # compared (both solutions meet the 1e-8 residual)
    assert rc == 0 and abs(it - it_ref) <= 2 and tr <= 1e-8
    from gpu_util import hist_atol
    np.testing.assert_allclose(hist[:15], h_ref[:15], rtol=1e-8, atol=hist_atol(1e-15))
    assert rel_err(P.to_ref(xs), u_ref) <= 1e-6
    N2 = Pair(mesh, n, lam, neumann=True, coarse=False)
    assert rel_err(N2.to_ref(N2.gpu.apply_P(N2.to_gpu(x), "fine")), N2.ref.apply_Pf(x)) <= TOL


def test_inverted_element_mesh_rejected():
    """A split-triangle mesh perturbed by 20 % has inverted corners: sem_create refuses it."""
    from paper_1506_05996_gb300 import sem
    from synth import split_triangle_hex_mesh
    mesh = split_triangle_hex_mesh(2, 2, a=0.2, seed=1)
    with pytest.raises(sem.SemError) as exc:
        sem.SemProblem(mesh.xyz, mesh.hex2vert, 3, 0.4)
    assert exc.value.code == sem.SEM_ERR_JACOBIAN


@pytest.mark.parametrize("geom", ["stored", "recompute"])
def test_random_mask_apply_parity(geom):
    """A Dirichlet set of random DOFs, element interiors included (sem_set_mask): y = A_D x
    against the oracle, where the element kernel writes interior DOFs of y itself (masked ones
    take x); FP32 within 2e-6 of the FP64 result."""
    from gpu_util import rel_err
    from paper_1506_05996_gb300 import sem
    mesh = lattice_hex_mesh(3, 0.2, 31)
    P = _pair(mesh, 5, 0.6, geom=geom, neumann=True, coarse=False)
    rng = np.random.default_rng(32)
    mask = (rng.random(P.ref.G) < 0.15).astype(np.uint8)
    mg = torch.zeros(P.gpu.n_dof, dtype=torch.uint8, device="cuda")
    mg[torch.as_tensor(P.perm, device="cuda")] = torch.as_tensor(mask, device="cuda")
    sem.sem_set_mask(P.gpu.h, mg)
    P.ref.mask = mask
    x = rng.standard_normal(P.ref.G)
    y64 = P.gpu.apply_A(P.to_gpu(x))
    assert rel_err(P.to_ref(y64), P.ref.apply_A(x)) <= TOL
    if geom == "recompute":
        P.gpu.set_precision("fp32")
        y32 = P.gpu.apply_A(P.to_gpu(x))
        assert rel_err(P.to_ref(y32), P.to_ref(y64)) <= 2e-6
        P.gpu.set_precision("fp64")
