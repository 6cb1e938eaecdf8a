"""ctypes binding of libsldm (the C ABI in ``include/sldm.h``), same names.

Argument marshalling only: numpy arrays are passed as host pointers and torch
CUDA tensors as device pointers (``where`` = SLDM_DEVICE).  The library must
have been built (``paper_2106_06184_gb300.build.build()``); there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsldm.so")

OK, EINVAL, ENOMEM, ENOTCONV, ENUMERIC, ECUDA, EBUSY, ENOTSUP, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8
INJECT_LU_STALL = 1
HOST, DEVICE = 0, 1
PREC_F64, PREC_F32, PREC_F32X2 = 0, 1, 2
BOTTOM_HALFSPACE, BOTTOM_PEC = 0, 1
(BLOCK_LAM, BLOCK_LPM, BLOCK_LA, BLOCK_LP, BLOCK_K, BLOCK_Y11, BLOCK_Y21, BLOCK_IX, BLOCK_KBAR_L) = range(9)


class SldmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sldm error {code}: {msg}")
        self.code = code


class Material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("mu_r", C.c_double), ("sigma", C.c_double),
                ("layer", C.c_int32), ("reserved", C.c_int32)]


class Layer(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("mu_r", C.c_double), ("sigma", C.c_double), ("thickness", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [("nv", C.c_int64), ("nt", C.c_int64), ("ne", C.c_int64), ("nobj", C.c_int64),
                ("n_unknowns", C.c_int64), ("n_bary_edges", C.c_int64)]


class AssembleOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("nested_min", C.c_int32), ("stream", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("x0_given", C.c_int32), ("precond", C.c_int32), ("refine", C.c_int32), ("reserved", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("relres", C.c_double)]


class OpInfo(C.Structure):
    _fields_ = [("n_unknowns", C.c_int64), ("ne", C.c_int64), ("nt", C.c_int64), ("nobj", C.c_int64),
                ("device_bytes", C.c_int64), ("precision", C.c_int32), ("tc_from", C.c_int32), ("k0", C.c_double)]


class ServerOpts(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_batch", C.c_int32), ("precision", C.c_int32), ("maxit", C.c_int32),
                ("budget_bytes", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("model", C.c_int32), ("nrhs", C.c_int32), ("freq_hz", C.c_double), ("khat", C.c_void_p),
                ("pol", C.c_void_p), ("tol", C.c_double), ("x", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("code", C.c_int32), ("iters", C.c_int32), ("relres", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("cache_hit", C.c_int32), ("batch_rhs", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("requests", C.c_int64), ("rhs", C.c_int64), ("batches", C.c_int64), ("hits", C.c_int64),
                ("misses", C.c_int64), ("evictions", C.c_int64), ("rejected", C.c_int64), ("cached_ops", C.c_int64),
                ("cached_bytes", C.c_int64), ("lat_p50", C.c_double), ("lat_p99", C.c_double), ("lat_max", C.c_double)]


EXPORTS = {
    "sldm_last_error": (None, [C.c_char_p, C.c_size_t]),
    "sldm_mesh_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "sldm_mesh_info_get": (C.c_int, [C.c_void_p, C.POINTER(MeshInfo)]),
    "sldm_mesh_edges": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sldm_mesh_destroy": (C.c_int, [C.c_void_p]),
    "sldm_stack_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.POINTER(C.c_void_p)]),
    "sldm_stack_destroy": (C.c_int, [C.c_void_p]),
    "sldm_assemble": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(AssembleOpts),
                                C.POINTER(C.c_void_p)]),
    "sldm_op_info_get": (C.c_int, [C.c_void_p, C.POINTER(OpInfo)]),
    "sldm_op_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sldm_op_destroy": (C.c_int, [C.c_void_p]),
    "sldm_op_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "sldm_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "sldm_rhs_planewave": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                     C.c_void_p]),
    "sldm_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(SolveOpts),
                             C.POINTER(SolveInfo), C.c_int32, C.c_void_p]),
    "sldm_farfield": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sldm_farfield_n": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                  C.c_void_p]),
    "sldm_kbar_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "sldm_timers_enable": (C.c_int, [C.c_int32]),
    "sldm_timers_reset": (C.c_int, []),
    "sldm_timer_get": (C.c_int, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "sldm_timer_names": (C.c_int, [C.c_char_p, C.c_size_t]),
    "sldm_launch_count": (C.c_int, [C.POINTER(C.c_int64)]),
    "sldm_timer_units": (C.c_int, [C.c_char_p, C.POINTER(C.c_double)]),
    "sldm_set_device_budget": (C.c_int, [C.c_int64]),
    "sldm_set_tc_policy": (C.c_int, [C.c_int32]),
    "sldm_device_bytes": (C.c_int, [C.POINTER(C.c_int64)]),
    "sldm_test_inject": (C.c_int, [C.c_int32, C.c_int32]),
    "sldm_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "sldm_server_add_model": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "sldm_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "sldm_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.POINTER(Result)]),
    "sldm_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "sldm_server_flush": (C.c_int, [C.c_void_p]),
    "sldm_server_destroy": (C.c_int, [C.c_void_p]),
    "sldm_cache_plan": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "sldm_batch_plan": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sldm_port_ring": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                 C.c_void_p, C.POINTER(C.c_int32)]),
    "sldm_port_rhs": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                C.c_void_p, C.c_int32, C.c_void_p]),
    "sldm_port_currents": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_int32, C.c_void_p]),
    "sldm_port_sparams": (C.c_int, [C.c_int32, C.c_void_p, C.c_double, C.c_void_p]),
}


class Library:
    """The loaded shared library with typed entry points."""

    def __init__(self, path=LIB_PATH):
        if not os.path.exists(path):
            raise SldmError(ENOTSUP, f"libsldm not built: {path} is missing (run paper_2106_06184_gb300.build)")
        self.path = path
        self.lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(self.lib, name)
            fn.restype = res
            fn.argtypes = args

    def check(self, code):
        if code != OK:
            buf = C.create_string_buffer(1024)
            self.lib.sldm_last_error(buf, 1024)
            raise SldmError(code, buf.value.decode(errors="replace"))
        return code


_LIB = None


def timers_enable(on=True, lib=None):
    L = lib or load()
    L.check(L.lib.sldm_timers_enable(int(bool(on))))


def timers_reset(lib=None):
    L = lib or load()
    L.check(L.lib.sldm_timers_reset())


def timers_read(lib=None):
    """{name: (total_ms, count)} of the library's timed launches."""
    L = lib or load()
    buf = C.create_string_buffer(4096)
    L.check(L.lib.sldm_timer_names(buf, 4096))
    out = {}
    for name in filter(None, buf.value.decode().split(",")):
        ms, n = C.c_double(), C.c_int64()
        L.check(L.lib.sldm_timer_get(name.encode(), C.byref(ms), C.byref(n)))
        out[name] = (ms.value, n.value)
    return out


def timer_units(name, lib=None) -> float:
    """sldm_timer_units: algorithmic units (bytes or evaluations) of the timed launches of `name`."""
    L = lib or load()
    v = C.c_double()
    L.check(L.lib.sldm_timer_units(name.encode(), C.byref(v)))
    return v.value


def launch_count(lib=None) -> int:
    """Kernel launches the library has made in this process."""
    L = lib or load()
    n = C.c_int64()
    L.check(L.lib.sldm_launch_count(C.byref(n)))
    return n.value


def set_tc_policy(tc_from=0, lib=None):
    """0: the tensor-core crossover is measured per operator; else forced."""
    L = lib or load()
    L.check(L.lib.sldm_set_tc_policy(int(tc_from)))


def set_device_budget(nbytes, lib=None):
    """sldm_set_device_budget: limit on the device bytes the library holds (0 = none)."""
    L = lib or load()
    L.check(L.lib.sldm_set_device_budget(int(nbytes)))


def device_bytes(lib=None) -> int:
    L = lib or load()
    v = C.c_int64()
    L.check(L.lib.sldm_device_bytes(C.byref(v)))
    return v.value


def test_inject(what, count, lib=None):
    """sldm_test_inject (failure-path tests)."""
    L = lib or load()
    L.check(L.lib.sldm_test_inject(int(what), int(count)))


def load(path=LIB_PATH) -> Library:
    global _LIB
    if _LIB is None or _LIB.path != path:
        _LIB = Library(path)
    return _LIB


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch CUDA tensor (device)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST)
    raise TypeError("expected a numpy array or a torch tensor")


def _stream(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Mesh:
    """sldm_mesh: closed outward-oriented triangle meshes, one or more objects."""

    h = None

    def __init__(self, xyz, tri, obj=None, lib=None):
        self.L = lib or load()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        objp = None
        if obj is not None:
            self._obj = np.ascontiguousarray(obj, dtype=np.int32)
            objp = self._obj.ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        self.L.check(self.L.lib.sldm_mesh_create(xyz.ctypes.data_as(C.c_void_p), len(xyz),
                                                 tri.ctypes.data_as(C.c_void_p), len(tri), objp, C.byref(h)))
        self.h = h
        info = MeshInfo()
        self.L.check(self.L.lib.sldm_mesh_info_get(h, C.byref(info)))
        self.nv, self.nt, self.ne, self.nobj = info.nv, info.nt, info.ne, info.nobj
        self.n_unknowns, self.n_bary_edges = info.n_unknowns, info.n_bary_edges

    def edges(self):
        uv = np.zeros((self.ne, 2), np.int64)
        tp = np.zeros(self.ne, np.int64)
        tm = np.zeros(self.ne, np.int64)
        self.L.check(self.L.lib.sldm_mesh_edges(self.h, uv.ctypes.data_as(C.c_void_p), tp.ctypes.data_as(C.c_void_p),
                                                tm.ctypes.data_as(C.c_void_p)))
        return uv, tp, tm

    def kbar_noalloc(self, obj, k, out, stream=None):
        """Kbar(k) of object `obj` into the device tensor `out` (ne_o x ne_o complex128)
        through the allocation-free entry point."""
        po, wo = _ptr(out)
        if wo != DEVICE:
            raise ValueError("kbar_noalloc writes device memory")
        self.L.check(self.L.lib.sldm_kbar_noalloc(self.h, obj, float(np.real(k)), float(np.imag(k)), po,
                                                  _stream(stream)))
        return out

    def close(self):
        if self.h:
            self.L.lib.sldm_mesh_destroy(self.h)
            self.h = None

    __del__ = close


class Stack:
    """sldm_stack: background layers listed top to bottom (one layer = homogeneous)."""

    h = None

    def __init__(self, layers, z_top=0.0, bottom=BOTTOM_HALFSPACE, lib=None):
        self.L = lib or load()
        arr = (Layer * len(layers))(*[Layer(*l) for l in layers])
        h = C.c_void_p()
        self.L.check(self.L.lib.sldm_stack_create(arr, len(layers), z_top, bottom, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.L.lib.sldm_stack_destroy(self.h)
            self.h = None

    __del__ = close


class Operator:
    """sldm_op: the assembled single-layer dual-mesh operator at one frequency."""

    h = None

    def __init__(self, mesh: Mesh, stack: Stack, materials, freq_hz, precision=PREC_F64, stream=None, nested_min=0):
        self.L = mesh.L
        self.mesh, self.stack = mesh, stack
        mats = (Material * len(materials))(*[Material(m[0], m[1], m[2], m[3] if len(m) > 3 else 0, 0)
                                             for m in materials])
        opts = AssembleOpts(precision, int(nested_min), _stream(stream))
        h = C.c_void_p()
        self.L.check(self.L.lib.sldm_assemble(mesh.h, stack.h, mats, freq_hz, C.byref(opts), C.byref(h)))
        self.h = h
        info = OpInfo()
        self.L.check(self.L.lib.sldm_op_info_get(h, C.byref(info)))
        self.N, self.ne, self.nt, self.nobj = info.n_unknowns, info.ne, info.nt, info.nobj
        self.k0, self.device_bytes, self.precision = info.k0, info.device_bytes, info.precision
        self.tc_from = info.tc_from

    def block(self, which, obj=0):
        r, c = C.c_int64(), C.c_int64()
        self.L.check(self.L.lib.sldm_op_block(self.h, which, obj, None, HOST, C.byref(r), C.byref(c)))
        out = np.zeros((r.value, c.value), np.complex128)
        self.L.check(self.L.lib.sldm_op_block(self.h, which, obj, out.ctypes.data_as(C.c_void_p), HOST,
                                              C.byref(r), C.byref(c)))
        return out

    def block_into(self, which, out, obj=0):
        """sldm_op_block into a caller buffer (numpy: host; torch CUDA tensor: device), complex128."""
        r, c = C.c_int64(), C.c_int64()
        self.L.check(self.L.lib.sldm_op_block(self.h, which, obj, None, HOST, C.byref(r), C.byref(c)))
        assert tuple(out.shape) == (r.value, c.value)
        p, w = _ptr(out)
        self.L.check(self.L.lib.sldm_op_block(self.h, which, obj, p, w, C.byref(r), C.byref(c)))
        return out

    def table(self, which):
        """Remainder table of a layered operator: (array (5, nr, n2), grid (5,))."""
        dims = (C.c_int64 * 3)()
        grid = (C.c_double * 5)()
        self.L.check(self.L.lib.sldm_op_table(self.h, which, None, dims, grid))
        out = np.zeros(tuple(dims), np.complex128)
        self.L.check(self.L.lib.sldm_op_table(self.h, which, out.ctypes.data_as(C.c_void_p), dims, grid))
        return out, np.array(list(grid))

    def apply(self, x, y, nrhs=1, stream=None):
        px, wx = _ptr(x)
        py, wy = _ptr(y)
        assert wx == wy
        self.L.check(self.L.lib.sldm_apply(self.h, px, py, nrhs, wx, _stream(stream)))
        return y

    def rhs_planewave(self, khat, pol, b, stream=None):
        khat = np.ascontiguousarray(np.atleast_2d(khat), np.float64)
        pol = np.ascontiguousarray(np.atleast_2d(pol), np.float64)
        pb, wb = _ptr(b)
        self.L.check(self.L.lib.sldm_rhs_planewave(self.h, khat.ctypes.data_as(C.c_void_p),
                                                   pol.ctypes.data_as(C.c_void_p), len(khat), pb, wb, _stream(stream)))
        return b

    def solve(self, b, x, nrhs=1, tol=1e-8, restart=300, maxit=2000, x0=False, precond=True, refine=True, stream=None,
              check=True):
        pb, wb = _ptr(b)
        px, wx = _ptr(x)
        assert wb == wx
        opts = SolveOpts(tol, restart, maxit, int(bool(x0)), 0 if precond else 1, 0 if refine else 1, 0)
        info = SolveInfo()
        code = self.L.lib.sldm_solve(self.h, pb, px, nrhs, C.byref(opts), C.byref(info), wb, _stream(stream))
        if check:
            self.L.check(code)
        return dict(iters=info.iters, relres=info.relres, status=info.status, code=code)

    def farfield(self, x, theta, phi):
        theta = np.ascontiguousarray(theta, np.float64)
        phi = np.ascontiguousarray(np.broadcast_to(phi, theta.shape), np.float64)
        out = np.zeros(len(theta))
        px, wx = _ptr(x)
        self.L.check(self.L.lib.sldm_farfield(self.h, px, wx, theta.ctypes.data_as(C.c_void_p),
                                              phi.ctypes.data_as(C.c_void_p), len(theta),
                                              out.ctypes.data_as(C.c_void_p)))
        return out

    def farfield_n(self, x, theta, phi, nrhs):
        """RCS of nrhs solutions x (nrhs, N) at once: (nrhs, len(theta))."""
        theta = np.ascontiguousarray(theta, np.float64)
        phi = np.ascontiguousarray(np.broadcast_to(phi, theta.shape), np.float64)
        out = np.zeros((nrhs, len(theta)))
        px, wx = _ptr(x)
        self.L.check(self.L.lib.sldm_farfield_n(self.h, px, nrhs, wx, theta.ctypes.data_as(C.c_void_p),
                                                phi.ctypes.data_as(C.c_void_p), len(theta),
                                                out.ctypes.data_as(C.c_void_p)))
        return out

    def port_rhs(self, ports, V, b, stream=None):
        """b (N x ncols per column, `where` of b) = sum_p V[p, k] port_p; V: (nports, ncols)."""
        V = np.ascontiguousarray(np.asarray(V, complex).reshape(ports.n, -1).T)  # column-major nports x ncols
        pb, wb = _ptr(b)
        self.L.check(self.L.lib.sldm_port_rhs(self.h, ports.n, *ports.args(), V.ctypes.data_as(C.c_void_p), V.shape[0],
                                              pb, wb, _stream(stream)))
        return b

    def port_currents(self, x, ports, ncols=1, stream=None):
        """Port currents (nports, ncols) of ncols solutions x."""
        out = np.zeros((ncols, ports.n), complex)  # column-major nports x ncols
        px, wx = _ptr(x)
        self.L.check(self.L.lib.sldm_port_currents(self.h, ports.n, *ports.args(), px, ncols,
                                                   out.ctypes.data_as(C.c_void_p), wx, _stream(stream)))
        return out.T.copy()

    def close(self):
        if self.h:
            self.L.lib.sldm_op_destroy(self.h)
            self.h = None

    __del__ = close


def port_ring(mesh, obj, s, c, tol=0.0):
    """(edges, signs) of the delta-gap port of object obj in the plane s . r = c."""
    L = mesh.L
    sv = np.ascontiguousarray(s, np.float64)
    n = C.c_int32(0)
    code = L.lib.sldm_port_ring(mesh.h, obj, sv.ctypes.data_as(C.c_void_p), c, tol, 0, None, None, C.byref(n))
    if n.value <= 0:
        L.check(code)
    edges = np.zeros(n.value, np.int32)
    signs = np.zeros(n.value, np.int8)
    L.check(L.lib.sldm_port_ring(mesh.h, obj, sv.ctypes.data_as(C.c_void_p), c, tol, n.value,
                                 edges.ctypes.data_as(C.c_void_p), signs.ctypes.data_as(C.c_void_p), C.byref(n)))
    return edges, signs


class Ports:
    """Several delta-gap ports as the CSR the C ABI takes: a list of (edges, signs)."""

    def __init__(self, rings):
        self.n = len(rings)
        self.ptr = np.zeros(self.n + 1, np.int32)
        self.ptr[1:] = np.cumsum([len(e) for e, _ in rings])
        self.edges = np.ascontiguousarray(np.concatenate([np.asarray(e, np.int32) for e, _ in rings]))
        self.signs = np.ascontiguousarray(np.concatenate([np.asarray(g, np.int8) for _, g in rings]))

    def args(self):
        return (self.ptr.ctypes.data_as(C.c_void_p), self.edges.ctypes.data_as(C.c_void_p),
                self.signs.ctypes.data_as(C.c_void_p))


def sparams(Y, z0=50.0, lib=None):
    """S = (1 - z0 Y)(1 + z0 Y)^-1 of an admittance matrix Y (n x n)."""
    L = lib or load()
    Y = np.atleast_2d(np.asarray(Y, complex))
    n = Y.shape[0]
    Yc = np.ascontiguousarray(Y.T)  # column-major
    out = np.zeros((n, n), complex)
    L.check(L.lib.sldm_port_sparams(n, Yc.ctypes.data_as(C.c_void_p), float(z0), out.ctypes.data_as(C.c_void_p)))
    return out.T.copy()


class Server:
    """sldm_server: the request loop over cached operators (argument marshalling only)."""

    h = None

    def __init__(self, workers=2, max_batch=32, precision=PREC_F32X2, budget_bytes=0, maxit=0, lib=None):
        self.L = lib or load()
        opts = ServerOpts(workers, max_batch, precision, maxit, int(budget_bytes))
        h = C.c_void_p()
        self.L.check(self.L.lib.sldm_server_create(C.byref(opts), C.byref(h)))
        self.h = h
        self._keep = {}  # ticket -> (khat, pol, x) kept alive until wait
        self._models = []

    def add_model(self, mesh, stack, materials):
        mats = (Material * len(materials))(*[Material(m[0], m[1], m[2], m[3] if len(m) > 3 else 0, 0)
                                             for m in materials])
        mid = C.c_int32()
        self.L.check(self.L.lib.sldm_server_add_model(self.h, mesh.h, stack.h, mats, C.byref(mid)))
        self._models.append((mesh, stack))
        return mid.value

    def submit(self, model, freq_hz, khat, pol, x, tol=1e-8):
        """x: host complex128 array (nrhs, N) receiving the solutions."""
        khat = np.ascontiguousarray(np.atleast_2d(khat), np.float64)
        pol = np.ascontiguousarray(np.atleast_2d(pol), np.float64)
        if not (isinstance(x, np.ndarray) and x.dtype == np.complex128 and x.flags.c_contiguous):
            raise ValueError("x must be a C-contiguous complex128 host array")
        req = Request(model, len(khat), freq_hz, khat.ctypes.data_as(C.c_void_p), pol.ctypes.data_as(C.c_void_p), tol,
                      x.ctypes.data_as(C.c_void_p))
        t = C.c_int64()
        self.L.check(self.L.lib.sldm_server_submit(self.h, C.byref(req), C.byref(t)))
        self._keep[t.value] = (khat, pol, x)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        r = Result()
        self.L.check(self.L.lib.sldm_server_wait(self.h, ticket, float(timeout), C.byref(r)))
        self._keep.pop(ticket, None)
        out = {f: getattr(r, f) for f, _ in Result._fields_}
        if r.code != OK:
            buf = C.create_string_buffer(1024)
            self.L.lib.sldm_last_error(buf, 1024)
            out["error"] = buf.value.decode(errors="replace")
        return out

    def stats(self):
        st = ServerStats()
        self.L.check(self.L.lib.sldm_server_stats_get(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def flush(self):
        self.L.check(self.L.lib.sldm_server_flush(self.h))

    def close(self):
        if self.h:
            self.L.lib.sldm_server_destroy(self.h)
            self.h = None

    __del__ = close


def cache_plan(keys, sizes, budget, lib=None):
    """The server's LRU admission policy on an access sequence: (action, evicted)."""
    L = lib or load()
    keys = np.ascontiguousarray(keys, np.int64)
    sizes = np.ascontiguousarray(sizes, np.int64)
    act = np.zeros(len(keys), np.int32)
    ev = np.zeros(len(keys), np.int32)
    L.check(L.lib.sldm_cache_plan(len(keys), keys.ctypes.data_as(C.c_void_p), sizes.ctypes.data_as(C.c_void_p),
                                  int(budget), act.ctypes.data_as(C.c_void_p), ev.ctypes.data_as(C.c_void_p)))
    return act, ev


def batch_plan(keys, nrhs, max_batch, lib=None):
    """The server's batching policy on a FIFO queue: the batch index of each request."""
    L = lib or load()
    keys = np.ascontiguousarray(keys, np.int64)
    nrhs = np.ascontiguousarray(nrhs, np.int32)
    out = np.zeros(len(keys), np.int32)
    L.check(L.lib.sldm_batch_plan(len(keys), keys.ctypes.data_as(C.c_void_p), nrhs.ctypes.data_as(C.c_void_p),
                                  int(max_batch), out.ctypes.data_as(C.c_void_p)))
    return out
