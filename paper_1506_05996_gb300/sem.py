"""Thin ctypes binding of libsem.so, one Python function per C entry point.

Only argument marshalling happens here: torch CUDA tensors become device
pointers, numpy arrays host pointers, and negative status codes become
SemError exceptions carrying sem_last_error(). Every step of the solver runs
in the library's CUDA kernels; if libsem.so is missing this module raises on
import.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsem.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libsem.so is not built (run `python -m paper_1506_05996_gb300.build`)")
_lib = ctypes.CDLL(LIB_PATH)

SEM_OK = 0
SEM_ERR_ARG, SEM_ERR_JACOBIAN, SEM_ERR_MESH, SEM_ERR_CUDA = -1, -2, -3, -4
SEM_ERR_OOM, SEM_ERR_NAN, SEM_ERR_SINGULAR = -5, -6, -7
SEM_MAXIT = 1
SEM_GEOM_STORED, SEM_GEOM_RECOMPUTE, SEM_NEUMANN, SEM_MIXED, SEM_PATCH_FULL = 0x0, 0x1, 0x10, 0x100, 0x1000
SEM_PREC_FP64, SEM_PREC_FP32, SEM_PREC_P32, SEM_PREC_BF16, SEM_PREC_FP64_NATIVE = 0, 1, 2, 3, 4
SEM_PRECOND_TWO_SCALE, SEM_PRECOND_FINE, SEM_PRECOND_NONE = 0, 1, 2
SEM_NET_LOSS_L2, SEM_NET_LOSS_ENERGY, SEM_NET_LOSS_ANGLE = 0, 1, 2
SEM_COARSE_VCYCLE, SEM_COARSE_KCYCLE = 0, 1
SEM_PATCH_SOLVE_FP32, SEM_PATCH_SOLVE_BF16_TC = 0, 1
SEM_LOOP_HOST, SEM_LOOP_DEVICE, SEM_LOOP_EAGER = 0, 1, 2

_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_P = ctypes.POINTER

_SIGS = {
    "sem_create": ([_vp, _i64, _vp, _i64, _int, _dbl, _int, _vp, _P(_vp)], _int),
    "sem_destroy": ([_vp], None),
    "sem_set_stream": ([_vp, _vp], _int),
    "sem_num_dofs": ([_vp, _P(_i64)], _int),
    "sem_num_elements": ([_vp, _P(_i64)], _int),
    "sem_dof_coords": ([_vp, _vp], _int),
    "sem_mass": ([_vp, _vp], _int),
    "sem_get_mask": ([_vp, _vp], _int),
    "sem_set_mask": ([_vp, _vp], _int),
    "sem_boundary_mask": ([_vp, _vp], _int),
    "sem_apply_mass": ([_vp, _vp, _vp], _int),
    "sem_coarse_levels": ([_vp, _int, _vp, _P(_int)], _int),
    "sem_apply_A": ([_vp, _vp, _vp], _int),
    "sem_apply_A_f32": ([_vp, _vp, _vp], _int),
    "sem_status": ([_vp], _int),
    "sem_apply_P": ([_vp, _vp, _vp], _int),
    "sem_apply_Pf": ([_vp, _vp, _vp], _int),
    "sem_apply_Pc": ([_vp, _vp, _vp], _int),
    "sem_set_precond": ([_vp, _int], _int),
    "sem_set_coarse_solver": ([_vp, _int], _int),
    "sem_set_loop": ([_vp, _int], _int),
    "sem_set_weights": ([_vp, _int], _int),
    "sem_set_patch_solver": ([_vp, _int], _int),
    "sem_set_overlap": ([_vp, _int], _int),
    "sem_set_precision": ([_vp, _int], _int),
    "sem_solve": ([_vp, _vp, _vp, _dbl, _int, _P(_int), _vp, _P(_dbl)], _int),
    "sem_apply_A_noalloc": ([_int, _i64, _i64, _dbl] + [_vp] * 8, _int),
    "sem_solve_many": ([_int, _vp, _vp, _vp, _dbl, _int, _vp, _vp], _int),
    "sem_solve_many_block": ([_int, _vp, _int, _vp, _vp, _dbl, _int, _vp, _vp], _int),
    "sem_solve_block": ([_vp, _int, _vp, _vp, _dbl, _int, _vp, _vp, _vp], _int),
    "sem_heat_step": ([_vp, _vp, _vp, _vp, _dbl, _int, _P(_int), _P(_dbl)], _int),
    "sem_set_tiles": ([_vp, _int, _int], _int),
    "sem_autotune": ([_vp, _P(_int), _P(_int)], _int),
    "sem_profile": ([_vp, _int], _int),
    "sem_selfcheck_convert": ([_vp, _i64, _P(_i64)], _int),
    "sem_measure_fma_peak": ([_int, _i64, _P(_dbl), _P(_dbl)], _int),
    "sem_profile_read": ([_vp, _int, _vp, _vp, _vp, _P(_int)], _int),
    "sem_net_create": ([ctypes.c_uint64, _P(_vp)], _int),
    "sem_net_destroy": ([_vp], None),
    "sem_net_num_params": ([], _int),
    "sem_net_get_params": ([_vp, _vp, _int], _int),
    "sem_net_set_params": ([_vp, _vp, _int], _int),
    "sem_net_apply": ([_vp, _vp, _vp, _vp], _int),
    "sem_net_pair": ([_vp] * 8, _int),
    "sem_net_gradient": ([_vp] * 6 + [_int, _vp, _P(_dbl)], _int),
    "sem_net_train_step": ([_vp] * 6 + [_int, ctypes.c_float, _P(_dbl)], _int),
    "sem_set_learned": ([_vp, _vp, _int, _dbl, _dbl], _int),
    "sem_learned_iterations": ([_vp, _P(_int)], _int),
    "sem_last_error": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class SemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libsem error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc < 0:
        raise SemError(rc, _lib.sem_last_error().decode())
    return rc


def _dev(t, dtype, n):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor of %s" % dtype)
    if t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def sem_last_error():
    return _lib.sem_last_error().decode()


def sem_create(vert_xyz, hex2vert, order, lam, flags=0, stream=None):
    xyz = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    hexes = np.ascontiguousarray(hex2vert, dtype=np.int64)
    if xyz.ndim != 2 or xyz.shape[1] != 3 or hexes.ndim != 2 or hexes.shape[1] != 8:
        raise ValueError("vert_xyz must be (n_vert, 3) and hex2vert (n_hex, 8)")
    h = ctypes.c_void_p()
    _check(_lib.sem_create(xyz.ctypes.data, xyz.shape[0], hexes.ctypes.data, hexes.shape[0],
                           int(order), float(lam), int(flags), _stream_ptr(stream), ctypes.byref(h)))
    return h


def sem_destroy(h):
    _lib.sem_destroy(h)


def sem_set_stream(h, stream):
    return _check(_lib.sem_set_stream(h, _stream_ptr(stream)))


def sem_num_dofs(h):
    n = ctypes.c_int64()
    _check(_lib.sem_num_dofs(h, ctypes.byref(n)))
    return n.value


def sem_num_elements(h):
    n = ctypes.c_int64()
    _check(_lib.sem_num_elements(h, ctypes.byref(n)))
    return n.value


def sem_dof_coords(h, xyz):
    return _check(_lib.sem_dof_coords(h, _dev(xyz, torch.float64, 3 * sem_num_dofs(h))))


def sem_mass(h, m):
    return _check(_lib.sem_mass(h, _dev(m, torch.float64, sem_num_dofs(h))))


def sem_get_mask(h, mask):
    return _check(_lib.sem_get_mask(h, _dev(mask, torch.uint8, sem_num_dofs(h))))


def sem_boundary_mask(h, mask):
    return _check(_lib.sem_boundary_mask(h, _dev(mask, torch.uint8, sem_num_dofs(h))))


def sem_apply_mass(h, s, b):
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_mass(h, _dev(s, torch.float64, n), _dev(b, torch.float64, n)))


def sem_coarse_levels(h, max_levels=32):
    sizes = np.zeros(max_levels, dtype=np.int64)
    n = ctypes.c_int()
    _check(_lib.sem_coarse_levels(h, max_levels, sizes.ctypes.data_as(_vp), ctypes.byref(n)))
    return [int(v) for v in sizes[:min(n.value, max_levels)]]


def sem_set_mask(h, mask):
    return _check(_lib.sem_set_mask(h, _dev(mask, torch.uint8, sem_num_dofs(h))))


def sem_apply_A_f32(h, x, y):
    """y = A x with FP32 CUDA tensors in and out (FP32 element arithmetic, no conversions)."""
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_A_f32(h, _dev(x, torch.float32, n), _dev(y, torch.float32, n)))


def sem_status(h):
    """Synchronise the handle's stream; raises if a kernel gave up a bounded barrier wait."""
    return _check(_lib.sem_status(h))


def sem_apply_A(h, x, y):
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_A(h, _dev(x, torch.float64, n), _dev(y, torch.float64, n)))


def sem_apply_P(h, r, z):
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_P(h, _dev(r, torch.float64, n), _dev(z, torch.float64, n)))


def sem_apply_Pf(h, r, z):
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_Pf(h, _dev(r, torch.float64, n), _dev(z, torch.float64, n)))


def sem_apply_Pc(h, r, z):
    n = sem_num_dofs(h)
    return _check(_lib.sem_apply_Pc(h, _dev(r, torch.float64, n), _dev(z, torch.float64, n)))


def sem_set_precond(h, which):
    return _check(_lib.sem_set_precond(h, int(which)))


def sem_set_coarse_solver(h, kind):
    return _check(_lib.sem_set_coarse_solver(h, {"vcycle": SEM_COARSE_VCYCLE, "kcycle": SEM_COARSE_KCYCLE}.get(kind, kind)))


def sem_set_overlap(h, reserve_sms):
    return _check(_lib.sem_set_overlap(h, int(reserve_sms)))


def sem_set_weights(h, weighted):
    return _check(_lib.sem_set_weights(h, int(bool(weighted))))


def sem_set_patch_solver(h, kind):
    k = {"fp32": SEM_PATCH_SOLVE_FP32, "bf16_tc": SEM_PATCH_SOLVE_BF16_TC}.get(kind, kind)
    return _check(_lib.sem_set_patch_solver(h, k))


def sem_set_loop(h, mode):
    return _check(_lib.sem_set_loop(h, {"host": SEM_LOOP_HOST, "device": SEM_LOOP_DEVICE,
                                        "eager": SEM_LOOP_EAGER}.get(mode, mode)))


def sem_set_precision(h, precision):
    return _check(_lib.sem_set_precision(h, int(precision)))


def sem_solve(h, b, x, rtol=1e-8, maxit=1000, want_history=True):
    """Returns (status, iterations, residual history (numpy) or None, true relative residual)."""
    n = sem_num_dofs(h)
    it = ctypes.c_int()
    tr = ctypes.c_double()
    hist = np.zeros(maxit + 1) if want_history else None
    rc = _check(_lib.sem_solve(h, _dev(b, torch.float64, n), _dev(x, torch.float64, n), float(rtol),
                               int(maxit), ctypes.byref(it), hist.ctypes.data if want_history else None,
                               ctypes.byref(tr)))
    if want_history:
        hist = hist[:it.value + 1].copy()
    return rc, it.value, hist, tr.value


def sem_apply_A_noalloc(order, n_hex, n_dof, lam, elem_xyz, l2g, g2l_off, g2l_idx, mask, x, y, stream=None):
    """y = A_D x with caller-owned tables and a static scratch array (no device allocation)."""
    p3 = (order + 1) ** 3
    args = [_dev(elem_xyz, torch.float64, 24 * n_hex), _dev(l2g, torch.int32, n_hex * p3),
            _dev(g2l_off, torch.int32, n_dof + 1), _dev(g2l_idx, torch.int32, n_hex * p3),
            _dev(mask, torch.uint8, n_dof), _dev(x, torch.float64, n_dof), _dev(y, torch.float64, n_dof)]
    return _check(_lib.sem_apply_A_noalloc(int(order), int(n_hex), int(n_dof), float(lam), *args,
                                           _stream_ptr(stream)))


def sem_heat_step(h, u_prev, g, u, rtol=1e-8, maxit=1000):
    """One backward-Euler step; returns (status, iterations, true relative residual)."""
    n = sem_num_dofs(h)
    it = ctypes.c_int()
    tr = ctypes.c_double()
    rc = _check(_lib.sem_heat_step(h, _dev(u_prev, torch.float64, n), _dev(g, torch.float64, n),
                                   _dev(u, torch.float64, n), float(rtol), int(maxit), ctypes.byref(it),
                                   ctypes.byref(tr)))
    return rc, it.value, tr.value


def sem_solve_many(handles, bs, xs, rtol=1e-8, maxit=1000):
    """Returns (status, iterations list, per-solve statuses)."""
    k = len(handles)
    H = (ctypes.c_void_p * k)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    ns = [sem_num_dofs(h) for h in handles]
    B = (ctypes.c_void_p * k)(*[_dev(b, torch.float64, n).value for b, n in zip(bs, ns)])
    X = (ctypes.c_void_p * k)(*[_dev(x, torch.float64, n).value for x, n in zip(xs, ns)])
    its = (ctypes.c_int * k)()
    sts = (ctypes.c_int * k)()
    rc = _check(_lib.sem_solve_many(k, ctypes.cast(H, ctypes.c_void_p), ctypes.cast(B, ctypes.c_void_p),
                                    ctypes.cast(X, ctypes.c_void_p), float(rtol), int(maxit),
                                    ctypes.cast(its, ctypes.c_void_p), ctypes.cast(sts, ctypes.c_void_p)))
    return rc, list(its), list(sts)


def sem_solve_block(h, b, x, rtol=1e-8, maxit=1000):
    """k solves at once: b and x are (k, N) contiguous CUDA float64 tensors. Returns
    (rc, iterations[k], status[k], true_rel_res[k])."""
    n = sem_num_dofs(h)
    if b.dim() != 2 or b.shape[1] != n or x.shape != b.shape:
        raise ValueError("b and x must be (k, %d)" % n)
    k = int(b.shape[0])
    its = np.zeros(k, dtype=np.int32)
    sts = np.zeros(k, dtype=np.int32)
    trs = np.zeros(k, dtype=np.float64)
    rc = _check(_lib.sem_solve_block(h, k, _dev(b, torch.float64, k * n), _dev(x, torch.float64, k * n),
                                     float(rtol), int(maxit), its.ctypes.data_as(_vp), sts.ctypes.data_as(_vp),
                                     trs.ctypes.data_as(_vp)))
    return rc, its.tolist(), sts.tolist(), trs.tolist()


def sem_solve_many_block(handles, bs, xs, rtol=1e-8, maxit=1000):
    """Block solves of several handles in one graph launch: bs[i], xs[i] are (k, N_i)
    contiguous CUDA float64 tensors with the same k. Returns (rc, iterations[i][k],
    status[i][k])."""
    c = len(handles)
    k = int(bs[0].shape[0]) if c else 1
    ns = [sem_num_dofs(h) for h in handles]
    for b, x, n in zip(bs, xs, ns):
        if b.dim() != 2 or b.shape != (k, n) or x.shape != b.shape:
            raise ValueError("every b and x must be (k, N) with the same k")
    H = (ctypes.c_void_p * c)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    B = (ctypes.c_void_p * c)(*[_dev(b, torch.float64, k * n).value for b, n in zip(bs, ns)])
    X = (ctypes.c_void_p * c)(*[_dev(x, torch.float64, k * n).value for x, n in zip(xs, ns)])
    its = np.zeros(c * k, dtype=np.int32)
    sts = np.zeros(c * k, dtype=np.int32)
    rc = _check(_lib.sem_solve_many_block(c, ctypes.cast(H, ctypes.c_void_p), k, ctypes.cast(B, ctypes.c_void_p),
                                          ctypes.cast(X, ctypes.c_void_p), float(rtol), int(maxit),
                                          its.ctypes.data_as(_vp), sts.ctypes.data_as(_vp)))
    return rc, its.reshape(c, k).tolist(), sts.reshape(c, k).tolist()


def sem_set_tiles(h, epb_ax, epb_sw):
    return _check(_lib.sem_set_tiles(h, int(epb_ax), int(epb_sw)))


def sem_autotune(h):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(_lib.sem_autotune(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sem_selfcheck_convert(bits):
    """Mismatches of the library's FP64 -> FP32 conversion against the GPU's, over the 64-bit
    patterns in `bits` (a CUDA int64 tensor)."""
    n = ctypes.c_int64()
    b = bits.contiguous()
    _check(_lib.sem_selfcheck_convert(ctypes.c_void_p(b.data_ptr()), int(b.numel()), ctypes.byref(n)))
    return n.value


def sem_measure_fma_peak(precision, iters):
    """(TFLOP/s, ms) of the library's FMA loop in FP64 ("fp64") or FP32 ("fp32")."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    prec = {"fp64": SEM_PREC_FP64, "fp32": SEM_PREC_FP32}[precision]
    _check(_lib.sem_measure_fma_peak(prec, int(iters), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def sem_profile(h, enable):
    return _check(_lib.sem_profile(h, int(bool(enable))))


def sem_profile_read(h, max_kernels=64):
    """Returns {kernel name: (launches, total milliseconds)}."""
    names = ctypes.create_string_buffer(64 * max_kernels)
    launches = np.zeros(max_kernels, dtype=np.int64)
    total = np.zeros(max_kernels)
    nk = ctypes.c_int()
    _check(_lib.sem_profile_read(h, max_kernels, ctypes.cast(names, ctypes.c_void_p), launches.ctypes.data,
                                 total.ctypes.data, ctypes.byref(nk)))
    out = {}
    for i in range(min(nk.value, max_kernels)):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(total[i]))
    return out


def sem_net_create(seed):
    net = ctypes.c_void_p()
    _check(_lib.sem_net_create(int(seed), ctypes.byref(net)))
    return net


def sem_net_destroy(net):
    _lib.sem_net_destroy(net)


def sem_net_num_params():
    return _lib.sem_net_num_params()


def sem_net_get_params(net):
    out = np.zeros(sem_net_num_params(), dtype=np.float32)
    _check(_lib.sem_net_get_params(net, out.ctypes.data, out.size))
    return out


def sem_net_set_params(net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    return _check(_lib.sem_net_set_params(net, a.ctypes.data, a.size))


def sem_net_apply(net, h, r, out):
    n = sem_num_dofs(h)
    return _check(_lib.sem_net_apply(net, h, _dev(r, torch.float64, n), _dev(out, torch.float64, n)))


def sem_net_pair(h, b, x_star, x_k, s, delta, r=None, z0=None):
    n = sem_num_dofs(h)
    opt = [None if v is None else _dev(v, torch.float64, n) for v in (r, z0)]
    return _check(_lib.sem_net_pair(h, *[_dev(v, torch.float64, n) for v in (b, x_star, x_k, s, delta)], *opt))


def sem_net_gradient(net, h, v, target, loss="energy", r=None, z0=None):
    """Returns (loss, gradient as float32 numpy array)."""
    n = sem_num_dofs(h)
    g = np.zeros(sem_net_num_params(), dtype=np.float32)
    out = ctypes.c_double()
    opt = [None if t is None else _dev(t, torch.float64, n) for t in (r, z0)]
    _check(_lib.sem_net_gradient(net, h, _dev(v, torch.float64, n), _dev(target, torch.float64, n), *opt,
                                 _LOSS[loss], g.ctypes.data, ctypes.byref(out)))
    return out.value, g


def sem_net_train_step(net, h, v, target, lr, loss="energy", r=None, z0=None):
    n = sem_num_dofs(h)
    out = ctypes.c_double()
    opt = [None if t is None else _dev(t, torch.float64, n) for t in (r, z0)]
    _check(_lib.sem_net_train_step(net, h, _dev(v, torch.float64, n), _dev(target, torch.float64, n), *opt,
                                   _LOSS[loss], float(lr), ctypes.byref(out)))
    return out.value


_LOSS = {"l2": SEM_NET_LOSS_L2, "energy": SEM_NET_LOSS_ENERGY, "angle": SEM_NET_LOSS_ANGLE}


def sem_set_learned(h, net, stall_window=8, stall_ratio=0.5, accept_theta=0.25):
    return _check(_lib.sem_set_learned(h, net, int(stall_window), float(stall_ratio), float(accept_theta)))


def sem_learned_iterations(h):
    n = ctypes.c_int()
    _check(_lib.sem_learned_iterations(h, ctypes.byref(n)))
    return n.value


class SemProblem:
    """Owns one handle; convenience wrappers returning torch tensors."""

    def __init__(self, mesh_xyz, hex2vert, order, lam, geom="stored", neumann=False, stream=None,
                 device="cuda", mixed=False, patch="face"):
        flags = SEM_GEOM_RECOMPUTE if geom == "recompute" else SEM_GEOM_STORED
        if patch == "full":
            flags |= SEM_PATCH_FULL
        if neumann:
            flags |= SEM_NEUMANN
        if mixed:
            flags |= SEM_MIXED
        self.device = torch.device(device)
        self.h = sem_create(mesh_xyz, hex2vert, order, lam, flags, stream)
        self.n_dof = sem_num_dofs(self.h)
        self.order = order

    def close(self):
        if self.h is not None:
            sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, dtype=torch.float64, n=None):
        return torch.empty(self.n_dof if n is None else n, dtype=dtype, device=self.device)

    def set_coarse_solver(self, kind):
        sem_set_coarse_solver(self.h, kind)

    def set_precision(self, prec):
        sem_set_precision(self.h, {"fp64": SEM_PREC_FP64, "fp32": SEM_PREC_FP32, "p32": SEM_PREC_P32,
                                   "bf16": SEM_PREC_BF16, "fp64_native": SEM_PREC_FP64_NATIVE}[prec])

    def dof_coords(self):
        x = self._vec(n=3 * self.n_dof)
        sem_dof_coords(self.h, x)
        return x.view(self.n_dof, 3)

    def mass(self):
        m = self._vec()
        sem_mass(self.h, m)
        return m

    def mask(self):
        m = self._vec(torch.uint8)
        sem_get_mask(self.h, m)
        return m

    def load(self, s):
        """b = m_N s on free DOFs, 0 on Dirichlet DOFs (sem_apply_mass)."""
        b = self._vec()
        sem_apply_mass(self.h, s, b)
        return b

    def apply_A(self, x):
        y = self._vec()
        sem_apply_A(self.h, x, y)
        return y

    def apply_P(self, r, part="two-scale"):
        z = self._vec()
        {"two-scale": sem_apply_P, "fine": sem_apply_Pf, "coarse": sem_apply_Pc}[part](self.h, r, z)
        return z

    def solve(self, b, rtol=1e-8, maxit=1000, precond="two-scale", x=None):
        sem_set_precond(self.h, {"two-scale": SEM_PRECOND_TWO_SCALE, "fine": SEM_PRECOND_FINE,
                                 "none": SEM_PRECOND_NONE}[precond])
        if x is None:
            x = self._vec()
        rc, it, hist, tr = sem_solve(self.h, b, x, rtol, maxit)
        return x, rc, it, hist, tr
