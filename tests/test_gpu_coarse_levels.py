"""The default coarse solver with aggregation levels above its dense one (Sec. 4.1,
Eq. coarse), on the GPU through the C ABI against the oracle: P^c and P within 1e-12,
PCG with the oracle's iteration count and history. Meshes of 26^3 and 30^3 hexes at
n = 2 give two smoothed-aggregation levels above the dense coarsest solve, so the
level kernels (fused restriction M, prolongation and post-smoothing N, Q) run as they
do in the 32^3 solves. Also the load b = m_N s (sem_apply_mass, Sec. 2.4) against the
oracle's, and sem_boundary_mask against the default mask."""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


@pytest.mark.parametrize("E,n,lam,neumann,seed", [(30, 2, 1.0, False, 3), (26, 2, 1.0, True, 5)])
def test_multilevel_vcycle_parity(E, n, lam, neumann, seed):
    from gpu_util import Pair, rel_err
    from paper_1506_05996_gb300 import sem
    P = Pair(lattice_hex_mesh(E, 0.2, seed), n, lam, neumann=neumann)
    sizes = P.ref.amg.sizes()
    assert len(P.ref.amg.levels) >= 2, sizes
    assert sem.sem_coarse_levels(P.gpu.h) == sizes
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(P.ref.G)
    rg = P.to_gpu(r)
    assert rel_err(P.to_ref(P.gpu.apply_P(rg, "coarse")), P.ref.apply_Pc(r)) <= TOL
    assert rel_err(P.to_ref(P.gpu.apply_P(rg, "two-scale")), P.ref.apply_P(r)) <= TOL
    # the load through the library (sem_apply_mass) against the oracle's
    s = manufactured_s(P.ref.coords, lam) + (0.3 * rng.standard_normal(P.ref.G) if neumann else 0.0)
    b_ref = P.ref.load(s)
    b = P.gpu.load(P.to_gpu(s))
    assert rel_err(P.to_ref(b), b_ref) <= 1e-14
    x, rc, it, hist, tr = P.gpu.solve(b, rtol=1e-8, maxit=500)
    u, it_ref, hist_ref = P.ref.solve(b_ref, rtol=1e-8, maxit=500)
    assert rc == 0 and it == it_ref, (it, it_ref)
    from gpu_util import hist_atol
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-9, atol=hist_atol(1e-14))
    assert rel_err(P.to_ref(x), u) <= 1e-10
    assert tr <= 1e-8


def test_apply_mass_and_boundary_mask():
    """b = m_N s on free DOFs and 0 on the Dirichlet ones, in place too; the boundary mask
    call returns the handle's mask."""
    from gpu_util import Pair, rel_err
    from paper_1506_05996_gb300 import sem
    P = Pair(lattice_hex_mesh(3, 0.2, 9), 4, 0.5, coarse=False, schwarz=False)
    s = np.random.default_rng(3).standard_normal(P.ref.G)
    sg = P.to_gpu(s)
    b = P.gpu.load(sg)
    assert rel_err(P.to_ref(b), P.ref.load(s)) <= 1e-14
    sem.sem_apply_mass(P.gpu.h, sg, sg)           # s and b may be one buffer
    assert torch.equal(sg, b)
    m1 = torch.zeros(P.gpu.n_dof, dtype=torch.uint8, device="cuda")
    sem.sem_boundary_mask(P.gpu.h, m1)
    assert torch.equal(m1, P.gpu.mask())
    np.testing.assert_array_equal(P.to_ref(m1), P.ref.mask)
