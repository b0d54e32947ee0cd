"""The device-driven solve loop (one graph with a while node per solve, one launch for a
batch) against the host-driven loop: same kernels in the same order, so solutions,
iteration counts and residual histories are bit-identical."""
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


def _run(prob, b, mode, maxit=1000):
    from paper_1506_05996_gb300 import sem
    sem.sem_set_loop(prob.h, mode)
    x = torch.empty_like(b)
    rc, it, hist, tr = sem.sem_solve(prob.h, b, x, 1e-8, maxit)
    return rc, it, hist, tr, x


@pytest.mark.parametrize("prec,coarse", [("fp64", "vcycle"), ("fp32", "vcycle"), ("fp64", "kcycle"),
                                         ("fp32", "kcycle")])
def test_device_loop_is_bit_identical_to_host_loop(prec, coarse):
    from paper_1506_05996_gb300.learn import make_problem
    prob, b = make_problem(12, 0.2, 31, 4, 1.0, mixed=True)
    prob.set_coarse_solver(coarse)
    prob.set_precision(prec)
    host = _run(prob, b, "host")
    dev = _run(prob, b, "device")
    again = _run(prob, b, "device")           # replay of the cached graph
    eager = _run(prob, b, "eager")            # the host loop without graphs
    for r in (dev, again, eager):
        assert r[0] == host[0] == 0 and r[1] == host[1]
        np.testing.assert_array_equal(r[2], host[2])
        assert torch.equal(r[4], host[4])
    prob.close()


def test_device_loop_with_network_and_maxit():
    from paper_1506_05996_gb300 import sem
    from paper_1506_05996_gb300.learn import make_problem
    prob, b = make_problem(8, 0.2, 32, 3, 0.5)
    net = sem.sem_net_create(4)
    theta = (np.random.default_rng(4).standard_normal(sem.sem_net_num_params()) * 0.05).astype(np.float32)
    sem.sem_net_set_params(net, theta)
    sem.sem_set_learned(prob.h, net)
    host = _run(prob, b, "host")
    used_host = sem.sem_learned_iterations(prob.h)
    dev = _run(prob, b, "device")
    assert dev[1] == host[1] and sem.sem_learned_iterations(prob.h) == used_host
    assert torch.equal(dev[4], host[4])
    sem.sem_set_learned(prob.h, None)
    sem.sem_net_destroy(net)
    # maxit reached inside the device loop: status, count and history as in the host loop
    h3 = _run(prob, b, "host", maxit=3)
    d3 = _run(prob, b, "device", maxit=3)
    assert h3[0] == d3[0] == sem.SEM_MAXIT and h3[1] == d3[1] == 3
    np.testing.assert_array_equal(d3[2], h3[2])
    prob.close()


def test_batched_single_launch_matches_single_solves():
    from paper_1506_05996_gb300 import sem
    from paper_1506_05996_gb300.learn import make_problem
    probs = [make_problem(E, 0.15, 40 + E, n, 0.0, load="gaussian", load_seed=E) for E, n in
             [(6, 3), (8, 5), (5, 7), (10, 2)]]
    singles = []
    for prob, b in probs:
        sem.sem_set_loop(prob.h, "host")
        x = torch.empty_like(b)
        rc, it, _, _ = sem.sem_solve(prob.h, b, x, 1e-8, 1000)
        singles.append((it, x))
        sem.sem_set_loop(prob.h, "device")
    xs = [torch.empty_like(b) for _, b in probs]
    for _ in range(2):                        # build, then replay the cached batch graph
        rc, its, sts = sem.sem_solve_many([p.h for p, _ in probs], [b for _, b in probs], xs, 1e-8, 1000)
        assert rc == 0 and all(s == 0 for s in sts)
        for (it, x), it2, x2 in zip(singles, its, xs):
            assert it2 == it and torch.equal(x2, x)
    for prob, _ in probs:
        prob.close()
