"""Block solves (sem_solve_block): k right-hand sides on one handle advanced together, every
kernel of an iteration one launch over all of them. Each right-hand side must give exactly the
result of its own sem_solve (same kernels on its slice, reductions over the same blocks in the
same order), converge independently (a converged or zero right-hand side stays put while the
others iterate), and match the oracle."""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


def _loads(P, k, seed):
    rng = np.random.default_rng(seed)
    free = P.ref.mask == 0
    bs = [P.ref.load(manufactured_s(P.ref.coords, P.ref.lam))]
    for _ in range(k - 1):
        bs.append(np.where(free, rng.standard_normal(P.ref.G), 0.0))
    return bs


@pytest.mark.parametrize("prec", ["fp64", "fp64_native"])
@pytest.mark.parametrize("E,n,lam,neumann,seed", [(4, 3, 0.0, False, 1), (3, 5, 1.0, False, 2),
                                                  (26, 2, 1.0, True, 5)])
def test_block_equals_single_solves(prec, E, n, lam, neumann, seed):
    from gpu_util import Pair, rel_err
    from paper_1506_05996_gb300 import sem
    P = Pair(lattice_hex_mesh(E, 0.2, seed), n, lam, neumann=neumann)
    P.gpu.set_precision(prec)
    k = 3
    bs = _loads(P, k, seed)
    B = torch.stack([P.to_gpu(b) for b in bs]).contiguous()
    X = torch.empty_like(B)
    rc, its, sts, trs = sem.sem_solve_block(P.gpu.h, B, X, 1e-8, 500)
    assert rc == 0 and all(s == 0 for s in sts)
    for j in range(k):
        x, rcj, it, hist, tr = P.gpu.solve(B[j].clone(), rtol=1e-8, maxit=500)
        assert rcj == 0 and it == its[j]
        assert torch.equal(x, X[j]), j            # bit-identical to the single solve
        assert tr == trs[j] and tr <= 1e-8
    # the first right-hand side against the oracle
    u, it_ref, _ = P.ref.solve(bs[0], rtol=1e-8, maxit=500)
    assert its[0] == it_ref
    assert rel_err(P.to_ref(X[0]), u) <= 1e-10


def test_block_right_hand_sides_converge_independently():
    from paper_1506_05996_gb300 import sem
    from gpu_util import Pair
    P = Pair(lattice_hex_mesh(4, 0.2, 3), 4, 0.5)
    bs = _loads(P, 4, 3)
    bs[2] = np.zeros(P.ref.G)                                # converged at the start
    bs[3] = bs[1] * 1e-6                                     # same direction, other scale
    B = torch.stack([P.to_gpu(b) for b in bs]).contiguous()
    X = torch.empty_like(B)
    rc, its, sts, trs = sem.sem_solve_block(P.gpu.h, B, X, 1e-8, 500)
    assert rc == 0 and its[2] == 0 and float(X[2].abs().max()) == 0.0
    assert its[0] > 0 and its[1] > 0 and its[3] > 0
    # a smaller maxit: some right-hand sides stop at it, the status says so per right-hand side
    rc, its2, sts2, _ = sem.sem_solve_block(P.gpu.h, B, X, 1e-8, 3)
    assert rc == sem.SEM_MAXIT and its2[0] == 3 and sts2[0] == sem.SEM_MAXIT and sts2[2] == 0
    # single solves on the same handle afterwards are unchanged
    x, rcs, it, hist, tr = P.gpu.solve(B[0].clone(), rtol=1e-8)
    assert rcs == 0 and it == its[0]


def test_block_refusals():
    from paper_1506_05996_gb300 import sem
    from paper_1506_05996_gb300.sem import SemProblem, SemError
    mesh = lattice_hex_mesh(2, 0.1, 4)
    pr = SemProblem(mesh.xyz, mesh.hex2vert, 3, 1.0, mixed=True)
    B = torch.zeros(2, pr.n_dof, dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    pr.set_precision("fp32")
    with pytest.raises(SemError):
        sem.sem_solve_block(pr.h, B, X)
    pr.set_precision("fp64")
    pr.set_coarse_solver(sem.SEM_COARSE_KCYCLE)
    with pytest.raises(SemError):
        sem.sem_solve_block(pr.h, B, X)
    pr.close()


def test_many_block_equals_block_solves():
    """sem_solve_many_block: several handles of different sizes and orders, k right-hand sides
    each, as branches of one graph launch; every column bit-identical to the handle's own
    sem_solve_block (the same kernels on the same slices), and a second launch of the cached
    graph again."""
    from paper_1506_05996_gb300 import sem
    from paper_1506_05996_gb300.sem import SemProblem
    specs = [(3, 3, 0.0, 11), (5, 2, 1.0, 12), (4, 5, 0.5, 13)]
    k = 4
    probs, Bs = [], []
    for E, n, lam, seed in specs:
        mesh = lattice_hex_mesh(E, 0.15, seed)
        pr = SemProblem(mesh.xyz, mesh.hex2vert, n, lam)
        free = (pr.mask() == 0).double()
        g = torch.Generator(device="cuda").manual_seed(seed)
        B = (torch.randn(k, pr.n_dof, dtype=torch.float64, device="cuda", generator=g) * free).contiguous()
        probs.append(pr)
        Bs.append(B)
    ref = []
    for pr, B in zip(probs, Bs):
        X = torch.empty_like(B)
        rc, its, sts, _ = sem.sem_solve_block(pr.h, B, X, 1e-8, 500)
        assert rc == 0
        ref.append((X, its))
    for _ in range(2):
        Xs = [torch.empty_like(B) for B in Bs]
        rc, its, sts = sem.sem_solve_many_block([pr.h for pr in probs], Bs, Xs, 1e-8, 500)
        assert rc == 0 and all(s == 0 for row in sts for s in row)
        for (Xr, itr), X, it in zip(ref, Xs, its):
            assert it == itr
            assert torch.equal(X, Xr)
    for pr in probs:
        pr.close()
