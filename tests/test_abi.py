"""The C-ABI library builds, loads and exports every symbol include/sem.h declares.
Argument checks that return before any CUDA call are exercised without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_05996_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-zA-Z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    import paper_1506_05996_gb300.sem as sem
    assert sorted(sem.EXPORTED) == declared_functions()


def test_argument_errors_without_gpu(lib):
    lib.sem_create.restype = ctypes.c_int
    lib.sem_last_error.restype = ctypes.c_char_p
    xyz = np.zeros((8, 3))
    hexes = np.arange(8, dtype=np.int64).reshape(1, 8)
    h = ctypes.c_void_p()
    for order in (0, 1, 9):
        rc = lib.sem_create(xyz.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(8),
                            hexes.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(1), ctypes.c_int(order),
                            ctypes.c_double(0.0), ctypes.c_int(0), None, ctypes.byref(h))
        assert rc == -1 and b"order" in lib.sem_last_error()
    rc = lib.sem_create(None, ctypes.c_int64(8), hexes.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(1),
                        ctypes.c_int(3), ctypes.c_double(0.0), ctypes.c_int(0), None, ctypes.byref(h))
    assert rc == -1
    rc = lib.sem_create(xyz.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(8),
                        hexes.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(1), ctypes.c_int(3),
                        ctypes.c_double(-1.0), ctypes.c_int(0), None, ctypes.byref(h))
    assert rc == -1 and b"lambda" in lib.sem_last_error()
    lib.sem_destroy(None)   # NULL is ignored
    lib.sem_num_dofs.restype = ctypes.c_int
    assert lib.sem_num_dofs(None, None) == -1
