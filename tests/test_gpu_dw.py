"""SEM_PREC_FP64's element kernels in double-FP32 (csrc/kdw.cuh) against the FP64 oracle.

Per-result bounds. A pair carries 48 significant bits, every step of the kernels errs by at
most 4 u^2 = 2^-46 of its operands' magnitudes (tests/test_dw_arith.py pins this on the
host), and binary64 inputs enter with a relative error below 2^-46. On the longest path of
a local operator result a value passes K = 4p + 16 such steps (the count of the FP32 bound),
so |y_dw - y| <= K 2^-46 |A|(|x|) (oracle.operator.matfree_abs); the patch solve passes
K = 6P + 24 steps, |z_dw - z| <= K 2^-46 |S||S^T|(|r|) (oracle.schwarz.apply_fine_abs).
binary64 itself errs by about K 2^-53 of the same magnitudes. The max-norm 1e-12 parity of
the other GPU tests holds for both arithmetics; the native binary64 kernels stay selectable
(SEM_PREC_FP64_NATIVE) and are checked here too.
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s

pytestmark = pytest.mark.gpu
U46 = 2.0 ** -46


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


def _pair(mesh, n, lam, **kw):
    from gpu_util import Pair
    return Pair(mesh, n, lam, **kw)


@pytest.mark.parametrize("E,n,lam,a,seed", [(2, 2, 0.3, 0.2, 0), (3, 3, 0.0, 0.2, 1), (2, 5, 1.0, 0.2, 2),
                                            (2, 7, 0.5, 0.2, 3), (2, 8, 2.0, 0.15, 4)])
def test_dw_operator_within_bound(E, n, lam, a, seed):
    from gpu_util import rel_err
    from oracle.operator import matfree_abs
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, coarse=False, schwarz=False)
    x = np.random.default_rng(seed).standard_normal(P.ref.G)
    y = P.ref.apply_A(x)
    ydw = P.to_ref(P.gpu.apply_A(P.to_gpu(x)))
    P.gpu.set_precision("fp64_native")
    y64 = P.to_ref(P.gpu.apply_A(P.to_gpu(x)))
    yabs = matfree_abs(x, P.ref.l2g, P.ref.Dh, P.ref.Gf, P.ref.m_loc, lam, P.ref.mask)
    free = P.ref.mask == 0
    K = 4 * (n + 1) + 16
    assert np.max(np.abs(ydw - y)[free] / (K * U46 * yabs[free])) <= 1.0
    assert rel_err(ydw, y) <= 1e-12 and rel_err(y64, y) <= 1e-12
    # masked rows are the identity in both
    assert np.array_equal(ydw[~free], x[~free]) and np.array_equal(y64[~free], x[~free])
    # the two arithmetics differ (the pair kernel really ran), by far less than the bound
    assert np.max(np.abs(ydw - y64)) > 0


@pytest.mark.parametrize("E,n,lam,a,seed", [(3, 2, 0.0, 0.2, 5), (2, 5, 1.0, 0.2, 6), (2, 7, 0.4, 0.2, 7),
                                            (2, 8, 1.5, 0.15, 8)])
def test_dw_fine_preconditioner_within_bound(E, n, lam, a, seed):
    from gpu_util import rel_err
    from oracle.schwarz import apply_fine_abs
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, coarse=False)
    r = np.random.default_rng(seed).standard_normal(P.ref.G)
    z = P.ref.apply_Pf(r)
    zdw = P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine"))
    P.gpu.set_precision("fp64_native")
    z64 = P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine"))
    zabs = apply_fine_abs(r, P.ref.ip, P.ref.S, P.ref.ev, P.ref.h, lam, P.ref.mask)
    free = P.ref.mask == 0
    K = 6 * (n + 3) + 24
    assert np.max(np.abs(zdw - z)[free] / (K * U46 * zabs[free])) <= 1.0
    assert rel_err(zdw, z) <= 1e-12 and rel_err(z64, z) <= 1e-12
    assert np.max(np.abs(zdw - z64)) > 0


def test_dw_natural_boundary_and_weighted_patches():
    """The plain (unfolded) pencils of insulated sides and the overlap weights in pairs."""
    from gpu_util import rel_err
    from oracle.problem import Problem
    from paper_1506_05996_gb300 import sem
    P = _pair(lattice_hex_mesh(3, 0.2, 9), 4, 0.7, neumann=True, coarse=False)
    r = np.random.default_rng(9).standard_normal(P.ref.G)
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine")), P.ref.apply_Pf(r)) <= 1e-12
    mesh = lattice_hex_mesh(3, 0.2, 10)
    Q = _pair(mesh, 5, 0.9, coarse=False)
    ref = Problem(mesh, 5, 0.9, coarse_solver=None, weights="cover")
    sem.sem_set_weights(Q.gpu.h, 1)
    r = np.random.default_rng(10).standard_normal(ref.G)
    assert rel_err(Q.to_ref(Q.gpu.apply_P(Q.to_gpu(r), "fine")), ref.apply_Pf(r)) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp64_native"])
def test_dw_and_native_solves_match_the_oracle(prec):
    """The same iteration count as the oracle and histories within 1e-9 in both arithmetics,
    and solutions within 1e-10 of each other."""
    from gpu_util import rel_err
    P = _pair(lattice_hex_mesh(6, 0.2, 11), 5, 1.0)
    b = P.ref.load(manufactured_s(P.ref.coords, 1.0))
    u, it_ref, hist_ref = P.ref.solve(b, rtol=1e-8)
    P.gpu.set_precision(prec)
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert rc == 0 and it == it_ref and tr <= 1e-8
    from gpu_util import hist_atol
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-9, atol=hist_atol(1e-14, prec))
    assert rel_err(P.to_ref(x), u) <= 1e-10


def test_dw_tiny_and_zero_inputs():
    """Inputs scaled by 2^-60 (pairs keep full precision down to 2^-80) and an all-zero x."""
    from gpu_util import rel_err
    P = _pair(lattice_hex_mesh(2, 0.2, 12), 4, 0.5, coarse=False)
    x = np.random.default_rng(12).standard_normal(P.ref.G) * 2.0 ** -60
    assert rel_err(P.to_ref(P.gpu.apply_A(P.to_gpu(x))), P.ref.apply_A(x)) <= 1e-12
    assert rel_err(P.to_ref(P.gpu.apply_P(P.to_gpu(x), "fine")), P.ref.apply_Pf(x)) <= 1e-12
    z = torch.zeros(P.gpu.n_dof, dtype=torch.float64, device="cuda")
    assert float(P.gpu.apply_A(z).abs().max()) == 0.0
