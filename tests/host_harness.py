"""Builds and loads tests/host_harness.cpp (the library's host set-up without CUDA)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "host_harness.cpp"),
       os.path.join(ROOT, "paper_1506_05996_gb300", "csrc", "host_setup.cpp"),
       os.path.join(ROOT, "paper_1506_05996_gb300", "csrc", "amg.cpp")]
OUT = os.path.join(ROOT, "paper_1506_05996_gb300", "_build", "host_harness.so")


def load():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(s) for s in SRC + [
            os.path.join(ROOT, "paper_1506_05996_gb300", "csrc", "host_setup.h")]):
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", OUT] + SRC, check=True)
    lib = ctypes.CDLL(OUT)
    lib.hh_G.restype = ctypes.c_int64
    return lib


class HostTables:
    def __init__(self, lib, mesh, n, lam, neumann=False, amg_kind=0, patch="face"):
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        hexes = np.ascontiguousarray(mesh.hex2vert, dtype=np.int64)
        rc = lib.hh_setup(xyz.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(xyz.shape[0]),
                          hexes.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(hexes.shape[0]),
                          ctypes.c_int(n), ctypes.c_double(lam), ctypes.c_int(int(neumann)),
                          ctypes.c_int(int(amg_kind)), ctypes.c_int(int(patch == "full")))
        self.rc = rc
        if rc != 0:
            return
        ne, p, P = hexes.shape[0], n + 1, n + 3
        self.G = lib.hh_G()
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self.l2g = np.zeros(ne * p ** 3, dtype=np.int32); lib.hh_l2g(vp(self.l2g))
        self.elem_perm = np.zeros(ne, dtype=np.int64); lib.hh_elem_perm(vp(self.elem_perm))
        self.g2l_off = np.zeros(self.G + 1, dtype=np.int32)
        self.g2l_idx = np.zeros(ne * p ** 3, dtype=np.int32)
        lib.hh_g2l(vp(self.g2l_off), vp(self.g2l_idx))
        self.coords = np.zeros(3 * self.G); lib.hh_coords(vp(self.coords))
        self.coords = self.coords.reshape(-1, 3)
        self.boundary = np.zeros(self.G, dtype=np.uint8); lib.hh_boundary(vp(self.boundary))
        self.ip = np.zeros(ne * P ** 3, dtype=np.int32); lib.hh_ip(vp(self.ip))
        self.hbox = np.zeros(ne * 3); lib.hh_hbox(vp(self.hbox))
        self.S = np.zeros(P * P); self.ev = np.zeros(P); lib.hh_pencil(vp(self.S), vp(self.ev))
        self.t = np.zeros(p); self.rho = np.zeros(p); self.D = np.zeros(p * p)
        lib.hh_gll(vp(self.t), vp(self.rho), vp(self.D))
        self.amg_sizes = [lib.hh_amg_size(l) for l in range(lib.hh_amg_nlevels() + 1)]
        self.nkeep = lib.hh_nkeep()
        self.keep = np.zeros(self.nkeep, dtype=np.int32); lib.hh_keep(vp(self.keep))
        self.lib = lib
        self.ne, self.p, self.P = ne, p, P

    def amg_matrix(self, l, which):
        """Level l's matrix as scipy CSR: 0 A, 1 P, 2 M, 3 N, 4 Q (the fused V-cycle)."""
        import scipy.sparse as sp
        n, m = self.lib.hh_amg_rows(l, which), self.lib.hh_amg_cols(l, which)
        nnz = self.lib.hh_amg_nnz(l, which)
        ptr = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self.lib.hh_amg_csr(l, which, vp(ptr), vp(col), vp(val))
        return sp.csr_matrix((val, col, ptr), shape=(n, m))

    def amg_level(self, l, which):
        n = self.amg_sizes[l]
        nnz = self.lib.hh_amg_nnz(l, which)
        ptr = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self.lib.hh_amg_csr(l, which, vp(ptr), vp(col), vp(val))
        return ptr, col, val

    def coarsest_inv(self):
        n = self.amg_sizes[-1]
        out = np.zeros(n * n)
        self.lib.hh_amg_coarsest(out.ctypes.data_as(ctypes.c_void_p))
        return out.reshape(n, n)
