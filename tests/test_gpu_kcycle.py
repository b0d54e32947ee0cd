"""The paper's coarse solver (Sec. 4.1): unsmoothed aggregation AMG applied as one
recursive K-cycle, under flexible PCG, on the GPU against the oracle.

The K-cycle is nonlinear but deterministic; P^c and P match at 1e-12, and the flexible
solve takes the oracle's iteration count with histories within 1e-7.
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def kp():
    from gpu_util import Pair
    return Pair(lattice_hex_mesh(24, 0.2, 11), 2, 0.7, kcycle=True)


def test_hierarchy_has_inner_kcycle_levels(kp):
    assert len(kp.ref.amg.levels) >= 2          # at least one level runs the inner flexible-CG steps


def test_coarse_and_two_scale_parity(kp):
    from gpu_util import rel_err
    rng = np.random.default_rng(1)
    r = rng.standard_normal(kp.ref.G) * (kp.ref.mask == 0)
    assert rel_err(kp.to_ref(kp.gpu.apply_P(kp.to_gpu(r), "coarse")), kp.ref.apply_Pc(r)) <= 1e-12
    assert rel_err(kp.to_ref(kp.gpu.apply_P(kp.to_gpu(r), "two-scale")), kp.ref.apply_P(r)) <= 1e-12
    # nonlinear: P(2 r) = 2 P(r) (homogeneous), but P(r + s) differs from P(r) + P(s)
    s = rng.standard_normal(kp.ref.G) * (kp.ref.mask == 0)
    a = kp.gpu.apply_P(kp.to_gpu(r + s), "coarse")
    b = kp.gpu.apply_P(kp.to_gpu(r), "coarse") + kp.gpu.apply_P(kp.to_gpu(s), "coarse")
    assert float((a - b).abs().max() / a.abs().max()) > 1e-8


def test_flexible_solve_parity(kp):
    from synth import manufactured_s
    b = kp.ref.load(manufactured_s(kp.ref.coords, kp.ref.lam))
    _, it_ref, h_ref = kp.ref.solve(b)
    x, rc, it, hist, tr = kp.gpu.solve(kp.to_gpu(b))
    assert rc == 0 and tr <= 1e-8
    assert it == it_ref
    from gpu_util import hist_atol
    np.testing.assert_allclose(hist, h_ref, rtol=1e-7, atol=hist_atol(1e-15))


def test_mixed_and_switch_back():
    from paper_1506_05996_gb300.learn import make_problem
    prob, b = make_problem(16, 0.2, 12, 4, 1.0, mixed=True)
    it_v = prob.solve(b)[2]
    prob.set_coarse_solver("kcycle")
    _, rc, it_k, _, tr = prob.solve(b)
    assert rc == 0 and tr <= 1e-8
    prob.set_precision("fp32")
    _, rc32, it_k32, _, tr32 = prob.solve(b)
    assert rc32 == 0 and tr32 <= 1e-8 and abs(it_k32 - it_k) <= 3
    prob.set_precision("fp64")
    prob.set_coarse_solver("vcycle")
    assert prob.solve(b)[2] == it_v
    prob.close()
