"""Backward-Euler heat steps (Sec. 5) on the GPU against oracle/heat.py.

Each library step solves for the increment from u_prev to rtol 1e-12 of the full
right-hand side; the fields after several steps match the oracle's direct solves to 1e-9
(relative, max-norm).
"""
import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh, moving_source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    build.build()


@pytest.mark.parametrize("neumann", [True, False])
def test_heat_steps_match_oracle(neumann):
    from gpu_util import Pair, rel_err
    from oracle.heat import HeatStepper
    from paper_1506_05996_gb300 import sem
    mesh = lattice_hex_mesh((2, 2, 6), 0.2, 5, box=(1.0, 1.0, 3.0))
    P = Pair(mesh, 4, 40.0, neumann=neumann, coarse=True)
    hs = HeatStepper(P.ref)
    free = P.ref.mask == 0
    u_ref = np.zeros(P.ref.G)
    u = torch.zeros(P.gpu.n_dof, dtype=torch.float64, device="cuda")
    for k in range(4):
        g = moving_source(P.ref.coords, 0.2 * k, q0=5.0, width=0.4) * free
        u_ref = hs.step(u_ref, g)
        rc, it, tr = sem.sem_heat_step(P.gpu.h, u, P.to_gpu(g), u, rtol=1e-12)
        assert rc == 0 and tr <= 1e-12 and it > 0
        assert rel_err(P.to_ref(u), u_ref) <= 1e-9, k


def test_heat_step_warm_start_and_mixed():
    from paper_1506_05996_gb300 import sem
    from paper_1506_05996_gb300.sem import SemProblem
    mesh = lattice_hex_mesh((3, 3, 9), 0.2, 6, box=(1.0, 1.0, 3.0))
    pr = SemProblem(mesh.xyz, mesh.hex2vert, 5, 100.0, neumann=True, mixed=True)
    X = pr.dof_coords().cpu().numpy()
    g = torch.as_tensor(moving_source(X, 0.0, q0=2.0), device="cuda")
    u = torch.zeros(pr.n_dof, dtype=torch.float64, device="cuda")
    its = []
    for _ in range(6):                      # a fixed source: the field approaches steady state
        rc, it, tr = sem.sem_heat_step(pr.h, u, g, u, rtol=1e-8)
        assert rc == 0 and tr <= 1e-8
        its.append(it)
    assert its[-1] < its[0]                 # the warm start needs fewer iterations as steps shrink
    u64 = u.clone()
    pr.set_precision("fp32")
    u32 = u.clone()
    rc, it32, tr32 = sem.sem_heat_step(pr.h, u32, g, u32, rtol=1e-8)
    pr.set_precision("fp64")
    rc, it64, tr64 = sem.sem_heat_step(pr.h, u64, g, u64, rtol=1e-8)
    assert tr32 <= 1e-8 and tr64 <= 1e-8
    assert float((u32 - u64).abs().max() / u64.abs().max()) <= 1e-7
    pr.close()
