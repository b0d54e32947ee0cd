"""Mixed-precision path (SEM_PREC_FP32) against the FP64 oracle.

Per-result bounds. The FP32 operator rounds x and the stored factors to FP32 and
forms every local result as nested sums of products, then sums the local copies of a
node (at most 8) in FP32; on the longest path a value passes K = 4p + 16 roundings
(p-term gradient, 3-term metric product, 3p-term divergence, the c-term, input
roundings, the gather), so |y32 - y| <= gamma_K u32 |A|(|x|) with u32 = 2^-24 and
|A|(|x|) the all-absolute apply (oracle.operator.matfree_abs). Recomputed geometry also rounds J, its cofactors and
|J| in FP32 (about 40 more roundings, amplified by the conditioning of J), so its bound
uses K = 4p + 8 + 40 kappa where kappa = max over nodes of cond(J)^2 (Frobenius),
computed by the oracle. The patch solve passes 6P + 4 roundings through |S| products and
the FP32 sum over the patches containing a node (at most 20 terms):
|z32 - z| <= gamma_{6P+24} u32 |S||S^T|(|r|) (oracle.schwarz.apply_fine_abs). The solve
must reach the FP64 true residual tolerance.
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, manufactured_s, manufactured_u

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def gamma(k):
    return k * U32 / (1 - k * U32)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


def _pair(mesh, n, lam, geom):
    from gpu_util import Pair
    P = Pair.__new__(Pair)
    from paper_1506_05996_gb300.sem import SemProblem
    from oracle.problem import Problem
    P.gpu = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom=geom, mixed=(geom == "stored"))
    P.ref = Problem(mesh, n, lam)
    Pair._match(P)
    return P


def _cond_J2(pr):
    from oracle.geometry import jacobians
    J = jacobians(pr.xyz_e, pr.t)
    c = np.linalg.norm(J, axis=(-2, -1)) * np.linalg.norm(np.linalg.inv(J), axis=(-2, -1))
    return float(np.max(c) ** 2)


@pytest.mark.parametrize("E,n,lam,a,seed", [(2, 3, 0.0, 0.2, 0), (3, 5, 1.0, 0.2, 1), (2, 7, 0.5, 0.2, 2),
                                            (2, 8, 2.0, 0.15, 3)])
@pytest.mark.parametrize("geom", ["stored", "recompute"])
def test_fp32_operator_within_bound(E, n, lam, a, seed, geom):
    from oracle.operator import matfree_abs
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, geom)
    x = np.random.default_rng(seed).standard_normal(P.ref.G)
    y64 = P.ref.apply_A(x)
    P.gpu.set_precision("fp32")
    y32 = P.to_ref(P.gpu.apply_A(P.to_gpu(x)))
    yabs = matfree_abs(x, P.ref.l2g, P.ref.Dh, P.ref.Gf, P.ref.m_loc, lam, P.ref.mask)
    p = n + 1
    K = 4 * p + 16 + (40 * _cond_J2(P.ref) if geom == "recompute" else 0)
    free = P.ref.mask == 0
    ratio = np.max(np.abs(y32 - y64)[free] / (gamma(K) * yabs[free]))
    assert ratio <= 1.0, ratio
    # and it is genuinely FP32 arithmetic, not FP64
    assert np.max(np.abs(y32 - y64)) > 0


U_BF16 = 2.0 ** -8


@pytest.mark.parametrize("E,n,lam,a,seed", [(2, 3, 0.0, 0.2, 0), (3, 5, 1.0, 0.2, 1), (2, 7, 0.5, 0.2, 2),
                                            (2, 8, 2.0, 0.15, 3)])
def test_bf16_operator_within_bound(E, n, lam, a, seed):
    """SEM_PREC_BF16: each stored factor is rounded once from FP64 to BF16 (relative error at
    most u_bf16 = 2^-8) and enters each product of the local result once, so on top of the
    FP32 bound |y16 - y| <= (u_bf16 (1 + gamma_K) + gamma_K) |A|(|x|)."""
    from oracle.operator import matfree_abs
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, "stored")
    x = np.random.default_rng(seed).standard_normal(P.ref.G)
    y64 = P.ref.apply_A(x)
    P.gpu.set_precision("bf16")
    y16 = P.to_ref(P.gpu.apply_A(P.to_gpu(x)))
    yabs = matfree_abs(x, P.ref.l2g, P.ref.Dh, P.ref.Gf, P.ref.m_loc, lam, P.ref.mask)
    K = 4 * (n + 1) + 16
    free = P.ref.mask == 0
    bound = (U_BF16 * (1 + gamma(K)) + gamma(K)) * yabs[free]
    ratio = np.max(np.abs(y16 - y64)[free] / bound)
    assert ratio <= 1.0, ratio
    # the factors really are BF16: the error exceeds the FP32 bound somewhere
    assert np.max(np.abs(y16 - y64)[free] / (gamma(K) * yabs[free])) > 1.0


def test_bf16_solve_is_refused():
    """The solves refuse SEM_PREC_BF16 (the mixed PCG with the BF16-factor operator stalls short of
    1e-8); FP32 then works on the same handle."""
    from paper_1506_05996_gb300.sem import SemError
    P = _pair(lattice_hex_mesh(4, 0.2, 4), 4, 1.0, "stored")
    b = P.ref.load(manufactured_s(P.ref.coords, 1.0))
    P.gpu.set_precision("bf16")
    with pytest.raises(SemError):
        P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    P.gpu.set_precision("fp32")
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert rc == 0 and tr <= 1e-8


def test_bf16_needs_stored_factors():
    from paper_1506_05996_gb300.sem import SemProblem, SemError
    mesh = lattice_hex_mesh(2, 0.1, 5)
    for kw in ({"geom": "recompute"}, {"geom": "stored"}):
        pr = SemProblem(mesh.xyz, mesh.hex2vert, 3, 1.0, **kw)
        with pytest.raises(SemError):
            pr.set_precision("bf16")
        pr.close()


@pytest.mark.parametrize("E,n,lam,a,seed", [(3, 3, 0.0, 0.2, 0), (2, 7, 1.0, 0.2, 1)])
def test_fp32_fine_preconditioner_within_bound(E, n, lam, a, seed):
    from oracle.schwarz import apply_fine_abs
    P = _pair(lattice_hex_mesh(E, a, seed), n, lam, "stored")
    r = np.random.default_rng(seed + 5).standard_normal(P.ref.G)
    z64 = P.ref.apply_Pf(r)
    P.gpu.set_precision("fp32")
    z32 = P.to_ref(P.gpu.apply_P(P.to_gpu(r), "fine"))
    zabs = apply_fine_abs(r, P.ref.ip, P.ref.S, P.ref.ev, P.ref.h, lam, P.ref.mask)
    K = 6 * (n + 3) + 24
    free = P.ref.mask == 0
    ratio = np.max(np.abs(z32 - z64)[free] / (gamma(K) * zabs[free]))
    assert ratio <= 1.0, ratio


@pytest.mark.parametrize("geom", ["stored", "recompute"])
def test_mixed_solve_reaches_fp64_tolerance(geom):
    P = _pair(lattice_hex_mesh(6, 0.2, 4), 5, 1.0, geom)
    b = P.ref.load(manufactured_s(P.ref.coords, 1.0))
    u_ref, it_ref, _ = P.ref.solve(b, rtol=1e-8)
    P.gpu.set_precision("fp32")
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert rc == 0
    assert tr <= 1e-8                      # the FP64 true residual, computed afresh
    assert it <= int(1.25 * it_ref) + 2
    u = P.to_ref(x)
    # both solutions satisfy ||b - A u|| <= 1e-8 ||b||; their difference is bounded by
    # 2e-8 ||b|| / lambda_min(A); compare against the manufactured-solution error scale
    assert np.max(np.abs(u - u_ref)) <= 1e-5 * np.max(np.abs(u_ref))
    assert np.max(np.abs(u - manufactured_u(P.ref.coords))) < 1e-3


def test_fp32_preconditioner_with_fp64_operator():
    """SEM_PREC_P32: the preconditioner alone in FP32, through the same kernels as the mixed
    path's FP32 P (so its results are bit-identical to them), with the FP64 operator: the
    recursive residual stays the FP64 one and the solve needs no replacement."""
    P = _pair(lattice_hex_mesh(6, 0.2, 4), 5, 1.0, "stored")
    rng = np.random.default_rng(11)
    r = P.to_gpu(rng.standard_normal(P.ref.G))
    P.gpu.set_precision("fp32")
    z_mixed = P.gpu.apply_P(r)
    P.gpu.set_precision("p32")
    z_p32 = P.gpu.apply_P(r)
    assert torch.equal(z_mixed, z_p32)
    b = P.ref.load(manufactured_s(P.ref.coords, 1.0))
    u_ref, it_ref, _ = P.ref.solve(b, rtol=1e-8)
    x, rc, it, hist, tr = P.gpu.solve(P.to_gpu(b), rtol=1e-8)
    assert rc == 0 and tr <= 1e-8 and abs(it - it_ref) <= 2
    # the recursive residual is the FP64 one: its last value agrees with the true residual
    assert abs(hist[-1] - tr) <= 1e-3 * tr
    u = P.to_ref(x)
    assert np.max(np.abs(u - u_ref)) <= 1e-5 * np.max(np.abs(u_ref))


def test_integer_conversion_matches_the_hardware():
    """The FP64 -> FP32 conversion the PCG vector kernels use (integer operations on the bit
    layouts) gives the bits of the conversion instruction: random patterns, every binary32
    exponent, ties and near-ties of the rounding, overflow, binary32 subnormals, zeros,
    infinities and NaNs."""
    from paper_1506_05996_gb300 import sem
    rng = np.random.default_rng(99)
    pats = [rng.integers(0, 2 ** 63, 1 << 20, dtype=np.int64) * np.where(rng.random(1 << 20) < 0.5, 1, -1)]
    # binary64 values near binary32 ones: f * (1 + k 2^-24) with k around +-1 (ties), at all exponents
    f = (rng.random(1 << 18) + 1.0) * np.exp2(rng.integers(-160, 130, 1 << 18)).astype(np.float64)
    with np.errstate(over="ignore"):
        f = f.astype(np.float32).astype(np.float64)
    for k in (-1.0, -1.0 + 2.0 ** -29, 1.0, 1.0 - 2.0 ** -29, 1.0 + 2.0 ** -29, 3.0, 0.5):
        pats.append((f * (1.0 + k * 2.0 ** -24)).view(np.int64))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.0 ** -149, 2.0 ** -150,
                        1.5 * 2.0 ** -150, 2.0 ** -126, 3.4028235677973366e38, 3.4028235677973362e38,
                        3.4028234663852886e38, 1e308, 2.0 ** -1022], dtype=np.float64).view(np.int64)
    pats.append(special)
    # every binary64 exponent that lands in or near the binary32 range, with several fractions
    ex = np.arange(800, 1300, dtype=np.int64)
    fr = np.array([0, 1, 1 << 28, (1 << 28) + 1, (1 << 29) - 1, 3 << 28, (1 << 52) - 1], dtype=np.int64)
    pats.append(((ex[:, None] << 52) | fr[None, :]).reshape(-1))
    bits = torch.as_tensor(np.concatenate(pats), device="cuda")
    assert sem.sem_selfcheck_convert(bits) == 0


@pytest.mark.parametrize("geom", ["stored", "recompute"])
def test_fp32_vector_apply_is_the_rounded_fp32_apply(geom):
    """sem_apply_A_f32 (FP32 vectors, no conversions) runs the same element and gather
    arithmetic as sem_apply_A in FP32 precision: for x exactly representable in FP32, its result
    agrees with that apply's to within 4 FP32 ulps of max|y| (a bound relative to the largest
    entry, not per entry: the compiler may contract the two instantiations differently);
    masked DOFs return x exactly."""
    from paper_1506_05996_gb300 import sem
    P = _pair(lattice_hex_mesh(3, 0.2, 7), 5, 0.7, geom)
    x32 = torch.randn(P.gpu.n_dof, dtype=torch.float32, device="cuda")
    P.gpu.set_precision("fp32")
    y64 = P.gpu.apply_A(x32.double())
    y32 = torch.empty_like(x32)
    sem.sem_apply_A_f32(P.gpu.h, x32, y32)
    scale = float(y64.abs().max())
    assert float((y32.double() - y64).abs().max()) <= 4 * 2.0 ** -24 * scale
    gm = torch.zeros(P.gpu.n_dof, dtype=torch.uint8, device="cuda")
    sem.sem_get_mask(P.gpu.h, gm)
    masked = gm.bool()
    assert bool(masked.any()) and torch.equal(y32[masked], x32[masked])
    assert sem.sem_status(P.gpu.h) == 0   # synchronises; no kernel gave up a bounded wait


@pytest.mark.parametrize("reserve", [None, -4])
def test_fp32_two_scale_on_a_capped_patch_grid(reserve):
    """The FP32 two-scale apply caps the patch-solve grid so that SMs stay free for the
    coarse branch, and its CTAs then loop over element groups. 32^3 hexes at n = 2 have
    more elements than any capped grid holds (at most (SMs - 48) x 32 resident CTAs of at
    most 8 elements), so the loop takes at least two rounds; reserve = -4 leaves only 4 SMs
    to the patch solves (many rounds). The fine part alone runs uncapped and is checked
    against the oracle's bound; the two-scale sum must then equal fine + coarse parts to one
    FP32 rounding (each patch result is computed by the same arithmetic in both launches)."""
    from oracle.schwarz import apply_fine_abs
    from paper_1506_05996_gb300 import sem
    E, n, lam = 32, 2, 1.0
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert E ** 3 > (nsm - 48) * 32 * 8
    P = _pair(lattice_hex_mesh(E, 0.2, 12), n, lam, "stored")
    P.gpu.set_precision("fp32")
    if reserve is not None:
        sem.sem_set_overlap(P.gpu.h, nsm + reserve)
    r = np.random.default_rng(13).standard_normal(P.ref.G)
    rg = P.to_gpu(r)
    zf = P.gpu.apply_P(rg, "fine")
    zc = P.gpu.apply_P(rg, "coarse")
    z = P.gpu.apply_P(rg, "two-scale")
    exact = zf + zc
    assert float((z - exact).abs().max()) <= 2.0 ** -23 * float(exact.abs().max())
    assert float((z - exact).abs().div(exact.abs() + 1e-300).max()) <= 2.0 ** -23
    zabs = apply_fine_abs(r, P.ref.ip, P.ref.S, P.ref.ev, P.ref.h, lam, P.ref.mask)
    K = 6 * (n + 3) + 24
    free = P.ref.mask == 0
    z64 = P.ref.apply_Pf(r)
    assert np.max(np.abs(P.to_ref(zf) - z64)[free] / (gamma(K) * zabs[free])) <= 1.0
