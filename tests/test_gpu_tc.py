"""BF16 patch solves of P^f on the tensor cores (sem_set_patch_solver(SEM_PATCH_SOLVE_BF16_TC),
csrc/k_swtc.cu) against the FP64 oracle.

Per-result bound. The box values, S and each of the six stages' inputs are rounded to BF16
(relative 2^-9 each, round to nearest), products are exact and accumulate in FP32 (at most
P terms, gamma_P u32), and the scaled modes are rounded once more: on the longest path a
value meets 13 BF16 roundings, so |z_tc - z| <= (13 2^-9 + 6 gamma_P) |S||S^T|(|r|)
(oracle.schwarz.apply_fine_abs) at every free node. The solves with it reach the FP64
true-residual tolerance (flexible PCG).
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
UB = 2.0 ** -9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


def _pair(mesh, n, lam):
    from gpu_util import Pair
    P = Pair.__new__(Pair)
    from paper_1506_05996_gb300.sem import SemProblem
    from oracle.problem import Problem
    P.gpu = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom="stored", mixed=True)
    P.ref = Problem(mesh, n, lam)
    Pair._match(P)
    return P


@pytest.mark.parametrize("E,n,lam,a,seed", [(3, 2, 0.0, 0.2, 0), (2, 3, 1.0, 0.2, 1), (3, 5, 0.5, 0.2, 2),
                                            (2, 7, 1.0, 0.2, 3), (2, 8, 2.0, 0.15, 4)])
@pytest.mark.parametrize("prec", ["fp32", "p32"])
def test_tc_fine_preconditioner_within_bound(E, n, lam, a, seed, prec):
    from oracle.schwarz import apply_fine_abs
    from paper_1506_05996_gb300 import sem
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam)
    r = np.random.default_rng(seed).standard_normal(P.ref.G)
    z64 = P.ref.apply_Pf(r)
    P.gpu.set_precision(prec)
    z32 = P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine"))
    sem.sem_set_patch_solver(P.gpu.h, "bf16_tc")
    ztc = P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine"))
    zabs = apply_fine_abs(r, P.ref.ip, P.ref.S, P.ref.ev, P.ref.h, lam, P.ref.mask)
    free = P.ref.mask == 0
    Pn = n + 3
    gP = Pn * U32 / (1 - Pn * U32)
    bound = (13 * UB + 6 * gP) * zabs[free]
    assert np.max(np.abs(ztc - z64)[free] / bound) <= 1.0
    # BF16 arithmetic really ran: the error is far above the FP32 kernel's
    assert np.max(np.abs(ztc - z64)[free]) > 100 * np.max(np.abs(z32 - z64)[free])
    assert np.all(ztc[~free] == 0.0)
    # deterministic
    assert np.array_equal(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), ztc)
    sem.sem_set_patch_solver(P.gpu.h, "fp32")
    assert np.array_equal(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), z32)


@pytest.mark.parametrize("reserve", [None, -4])
def test_tc_two_scale_on_a_capped_grid(reserve):
    """Beside the coarse branch the tensor-core CTAs loop over element groups on a capped grid;
    the two-scale sum equals fine + coarse parts to one FP32 rounding."""
    from paper_1506_05996_gb300 import sem
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    P = _pair(lattice_hex_mesh(20, 0.2, 5), 3, 1.0)
    assert 20 ** 3 > (nsm - 32) * 4 * 8        # more elements than one round of the capped grid
    P.gpu.set_precision("fp32")
    sem.sem_set_patch_solver(P.gpu.h, "bf16_tc")
    if reserve is not None:
        sem.sem_set_overlap(P.gpu.h, nsm + reserve)
    rg = P.to_gpu(np.random.default_rng(6).standard_normal(P.ref.G))
    zf, zc, z = P.gpu.apply_P(rg, "fine"), P.gpu.apply_P(rg, "coarse"), P.gpu.apply_P(rg, "two-scale")
    exact = zf + zc
    assert float((z - exact).abs().div(exact.abs() + 1e-300).max()) <= 2.0 ** -23


@pytest.mark.parametrize("prec", ["fp32", "p32"])
def test_tc_solve_reaches_fp64_tolerance(prec):
    from paper_1506_05996_gb300 import sem
    P = _pair(lattice_hex_mesh(6, 0.2, 7), 5, 1.0)
    b = P.ref.load(manufactured_s(P.ref.coords, 1.0))
    u_ref, it_ref, _ = P.ref.solve(b, rtol=1e-8)
    P.gpu.set_precision(prec)
    sem.sem_set_patch_solver(P.gpu.h, "bf16_tc")
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert rc == 0 and tr <= 1e-8
    assert it <= int(1.3 * it_ref) + 3, (it, it_ref)
    u = P.to_ref(x)
    assert np.max(np.abs(u - u_ref)) <= 1e-5 * np.max(np.abs(u_ref))
    # repeated solves are bit-identical
    x2, rc2, it2, hist2, tr2 = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert it2 == it and np.array_equal(hist2, hist)


def test_tc_natural_boundary_keeps_fp32_kernel():
    """Insulated faces take per-element pencils: the FP32 kernel serves the handle (results
    equal to the FP32 setting)."""
    from gpu_util import Pair
    from paper_1506_05996_gb300 import sem
    P = Pair(lattice_hex_mesh(3, 0.2, 8), 4, 0.7, neumann=True, coarse=False)
    P.gpu.set_precision("p32")
    r = P.to_gpu(np.random.default_rng(8).standard_normal(P.ref.G))
    z32 = P.gpu.apply_P(r, "fine")
    sem.sem_set_patch_solver(P.gpu.h, "bf16_tc")
    assert torch.equal(P.gpu.apply_P(r, "fine"), z32)
