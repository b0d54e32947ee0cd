"""sem_apply_A_noalloc against sem_apply_A, through the C ABI.

sem_apply_A_noalloc serves callers that cannot allocate device memory (code
running during stream capture, components whose memory a host framework hands
out, loops where allocator calls are not allowed): they pass every table and
vector, and the library's only scratch is a static device array of
SEM_NOALLOC_MAX_LOCAL_NODES doubles. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import lattice_hex_mesh

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 parity tolerance of the other operator tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05996_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.sem_apply_A_noalloc.restype = ctypes.c_int
    lib.sem_apply_A_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_double] + \
        [ctypes.c_void_p] * 8
    lib.sem_last_error.restype = ctypes.c_char_p
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_apply_A_on_two_calls(lib):
    from paper_1506_05996_gb300.sem import SemProblem
    from host_harness import load, HostTables
    mesh = lattice_hex_mesh(6, 0.2, 3)
    n, lam = 5, 0.7
    prob = SemProblem(mesh.xyz, mesh.hex2vert, n, lam, geom="recompute")
    # the host harness runs the library's own numbering code: same tables as the handle
    H = HostTables(load(), mesh, n, lam)
    assert H.rc == 0 and H.G == prob.n_dof
    np.testing.assert_array_equal(prob.dof_coords().cpu().numpy(), H.coords)
    dev = "cuda"
    exyz = torch.as_tensor(np.ascontiguousarray(mesh.xyz[mesh.hex2vert[H.elem_perm]]), device=dev)
    l2g = torch.as_tensor(H.l2g, device=dev)
    off = torch.as_tensor(H.g2l_off, device=dev)
    idx = torch.as_tensor(H.g2l_idx, device=dev)
    mask = prob.mask()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(0)
    for call in range(2):
        x = torch.as_tensor(rng.standard_normal(prob.n_dof), device=dev)
        y_ref = prob.apply_A(x)
        y = torch.full_like(x, float("nan"))
        rc = lib.sem_apply_A_noalloc(n, mesh.n_hex, prob.n_dof, lam, _ptr(exyz), _ptr(l2g), _ptr(off), _ptr(idx),
                                     _ptr(mask), _ptr(x), _ptr(y), ctypes.c_void_p(stream))
        assert rc == 0, lib.sem_last_error()
        torch.cuda.synchronize()
        err = float((y - y_ref).abs().max() / y_ref.abs().max())
        assert err <= TOL, (call, err)
    prob.close()


def test_noalloc_rejects_oversize(lib):
    from paper_1506_05996_gb300.sem import SEM_ERR_ARG
    n = 7
    n_hex = 2097152 // 512 + 1          # one element more than the static scratch holds
    dummy = ctypes.c_void_p(1)
    rc = lib.sem_apply_A_noalloc(n, n_hex, 1000, 0.0, dummy, dummy, dummy, dummy, dummy, dummy,
                                 ctypes.c_void_p(2), None)
    assert rc == SEM_ERR_ARG
    assert b"exceeds the static scratch" in lib.sem_last_error()
