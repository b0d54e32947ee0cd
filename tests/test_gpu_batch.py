"""Tile shapes and batched solves (the batched multi-problem launch)."""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, gaussian_load

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


@pytest.mark.parametrize("n", [3, 5, 8])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_tile_shapes_are_bit_identical(n, prec):
    from paper_1506_05996_gb300 import sem as S
    mesh = lattice_hex_mesh(5, 0.15, 3)     # 125 elements: short last CTAs for every shape
    pr = S.SemProblem(mesh.xyz, mesh.hex2vert, n, 0.5, mixed=True)
    pr.set_precision(prec)
    x = torch.randn(pr.n_dof, dtype=torch.float64, device="cuda")
    ref_y, ref_z = pr.apply_A(x), pr.apply_P(x, "fine")
    done = 0
    for epb in (2, 4, 8):
        try:
            S.sem_set_tiles(pr.h, epb, epb)
        except S.SemError:
            continue
        assert torch.equal(pr.apply_A(x), ref_y)
        assert torch.equal(pr.apply_P(x, "fine"), ref_z)
        done += 1
    if n <= 5:
        assert done >= 1
    a, b = S.sem_autotune(pr.h)
    assert a in (1, 2, 4, 8) and b in (1, 2, 4, 8)
    assert torch.equal(pr.apply_A(x), ref_y)
    pr.close()


def test_solve_many_equals_single_solves():
    from paper_1506_05996_gb300 import sem as S
    specs = [(4, 3), (6, 5), (5, 4), (3, 7)]
    probs, bs = [], []
    for k, (E, n) in enumerate(specs):
        mesh = lattice_hex_mesh(E, 0.15, 10 + k)
        st = torch.cuda.Stream()
        pr = S.SemProblem(mesh.xyz, mesh.hex2vert, n, 0.0, stream=st)
        m = pr.mask()
        b = torch.as_tensor(gaussian_load(pr.n_dof, 100 + k), device="cuda") * (m == 0)
        probs.append(pr)
        bs.append(b.contiguous())
    torch.cuda.synchronize()
    singles = []
    for pr, b in zip(probs, bs):
        x = torch.empty_like(b)
        rc, it, hist, tr = S.sem_solve(pr.h, b, x, 1e-8, 500, want_history=False)
        assert rc == 0
        singles.append((x.clone(), it))
    xs = [torch.empty_like(b) for b in bs]
    rc, its, sts = S.sem_solve_many([p.h for p in probs], bs, xs, 1e-8, 500)
    assert rc == 0 and all(s == 0 for s in sts)
    for (xs1, it1), x, it in zip(singles, xs, its):
        assert it == it1
        assert torch.equal(x, xs1)           # same kernels, same order: bit-identical
    for p in probs:
        p.close()
