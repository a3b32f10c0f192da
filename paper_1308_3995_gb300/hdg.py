"""Thin Python binding of the C ABI in ``include/hdg.h`` (argument marshalling
only; every step of the hot path runs in the CUDA library ``libhdg.so``).

Names follow the C functions: ``hdg_create`` -> :class:`Context`,
``hdg_mesh_create`` -> :class:`Mesh`, ``hdg_sys_create`` -> :class:`System`
with ``condense``/``recover``/``step_host``.  Device arrays are torch CUDA
tensors (plumbing for memory and streams); outputs are zero-copy torch views
of the library-owned buffers.  There is no CPU fallback: if the library cannot
be built or loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

HDG_OK, HDG_EINVAL, HDG_ENOMEM, HDG_ECUDA, HDG_ESINGULAR, HDG_ETIMEOUT, HDG_ENOTSUP = range(7)
HDG_EULER, HDG_NS_MIXED = 0, 1
HDG_FP64, HDG_FLOAT2, HDG_MIXED_TF32, HDG_MIXED_BF16 = 0, 1, 2, 3
STATUS_NAMES = {0: "HDG_OK", 1: "HDG_EINVAL", 2: "HDG_ENOMEM", 3: "HDG_ECUDA", 4: "HDG_ESINGULAR",
                5: "HDG_ETIMEOUT", 6: "HDG_ENOTSUP"}

# every entry point declared in include/hdg.h
EXPORTS = ["hdg_create", "hdg_destroy", "hdg_last_error", "hdg_mesh_create", "hdg_mesh_destroy", "hdg_mesh_sizes",
           "hdg_mesh_layout", "hdg_footprint_bytes", "hdg_sys_create", "hdg_sys_destroy", "hdg_condense",
           "hdg_recover", "hdg_step_host", "hdg_sys_get", "hdg_sys_launches", "hdg_debug_tables",
           "hdg_condense_noalloc", "hdg_sys_workspace_bytes", "hdg_sys_create_in",
           "hdg_step_host_async", "hdg_graph_create", "hdg_graph_launch", "hdg_solver_create",
           "hdg_solver_destroy", "hdg_trace_solve", "hdg_trace_matvec", "hdg_newton_update", "hdg_residual_norm",
           "hdg_sys_set_cfl", "hdg_cfl_law", "hdg_autotune", "hdg_trace_solve_ex", "hdg_adjoint_condense",
           "hdg_adapt_indicators", "hdg_adapt_mark",
           "hdg_mesh_create_bc", "hdg_solver_set_preconditioner", "hdg_solver_setup", "hdg_solver_precond_apply",
           "hdg_solver_colors", "hdg_solver_create_ws", "hdg_solver_workspace_bytes",
           "hdg_solver_create_ws_arith", "hdg_solver_workspace_bytes_arith", "hdg_solve_step_host",
           "hdg_sys_bucket_times", "hdg_sys_set_source", "hdg_batch_create", "hdg_batch_destroy",
           "hdg_batch_groups", "hdg_batch_condense", "hdg_batch_recover", "hdg_batch_step_host_async",
           "hdg_batch_autotune", "hdg_batch_graph_create", "hdg_batch_graph_launch", "hdg_batch_launches",
           "hdg_sys_io", "hdg_batch_workspace_bytes", "hdg_batch_create_in", "hdg_solver_set_arithmetic"]


class HdgError(RuntimeError):
    """A non-OK hdg_status with the library's last error message; ``status`` holds the code."""

    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class hdg_params(ctypes.Structure):
    """The C struct hdg_params (include/hdg.h), field for field."""
    _fields_ = [("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("reynolds", ctypes.c_double), ("mach", ctypes.c_double),
                ("alpha", ctypes.c_double), ("cfl", ctypes.c_double), ("t_inf", ctypes.c_double),
                ("refine_tol", ctypes.c_double), ("refine_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sc_eps0", ctypes.c_double), ("sc_beta", ctypes.c_double), ("aoa", ctypes.c_double)]


@dataclass
class Params:
    """Physical and numerical parameters of a system (hdg_params): model, arithmetic, gas
    constants, Mach number, stabilisation alpha, pseudo-time CFL (<= 0: pure Newton), shock
    capturing and the free-stream angle of attack."""
    model: int = HDG_EULER
    precision: int = HDG_FP64
    gamma: float = 1.4
    prandtl: float = 0.72
    reynolds: float = 5000.0
    mach: float = 0.5
    alpha: float = 1.5
    cfl: float = 0.0
    t_inf: float = 288.15
    refine_tol: float = 1e-13
    refine_max: int = 4
    sc_eps0: float = 0.0     # shock capturing (Sec. 3.2) off unless > 0 (paper's value 0.2)
    sc_beta: float = 0.0
    aoa: float = 0.0         # free-stream angle of attack [degrees]: the far-field state

    def c(self) -> hdg_params:
        """The C struct for a call."""
        return hdg_params(self.model, self.precision, self.gamma, self.prandtl, self.reynolds, self.mach,
                          self.alpha, self.cfl, self.t_inf, self.refine_tol, self.refine_max, 0,
                          self.sc_eps0, self.sc_beta, self.aoa)


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib(build: bool = True):
    """Load ``libhdg.so`` (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise HdgError(HDG_ENOTSUP, f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        L.hdg_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        L.hdg_destroy.argtypes = [_vp]
        L.hdg_last_error.argtypes = [_vp]
        L.hdg_last_error.restype = ctypes.c_char_p
        L.hdg_mesh_create.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _dp, _i32p,
                                      ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(_vp)]
        L.hdg_mesh_create_bc.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _dp, _i32p,
                                         ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int8),
                                         ctypes.POINTER(_vp)]
        L.hdg_mesh_destroy.argtypes = [_vp]
        L.hdg_mesh_sizes.argtypes = [_vp, _i64p]
        L.hdg_mesh_layout.argtypes = [_vp, _i32p, _i32p, _i32p, _i32p, _i64p, _i64p, _i64p, _i32p, _i64p]
        L.hdg_footprint_bytes.argtypes = [_vp, ctypes.POINTER(hdg_params)]
        L.hdg_footprint_bytes.restype = ctypes.c_int64
        L.hdg_sys_create.argtypes = [_vp, _vp, ctypes.POINTER(hdg_params), ctypes.POINTER(_vp)]
        L.hdg_sys_destroy.argtypes = [_vp]
        L.hdg_condense.argtypes = [_vp, _vp, _vp, _vp]
        L.hdg_recover.argtypes = [_vp, _vp, _vp, _vp]
        L.hdg_step_host.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.hdg_step_host_async.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.hdg_graph_create.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.hdg_graph_launch.argtypes = [_vp, _vp]
        L.hdg_sys_get.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 6
        L.hdg_sys_launches.argtypes = [_vp]
        L.hdg_sys_launches.restype = ctypes.c_int32
        L.hdg_debug_tables.argtypes = [ctypes.c_int] * 5 + [_dp, ctypes.c_int]
        L.hdg_condense_noalloc.argtypes = [_vp, ctypes.POINTER(hdg_params)] + [_vp] * 9
        L.hdg_batch_create.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]
        L.hdg_batch_destroy.argtypes = [_vp]
        L.hdg_batch_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp)]
        L.hdg_batch_workspace_bytes.restype = ctypes.c_int64
        L.hdg_batch_create_in.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(_vp), _vp, ctypes.c_int64, _vp,
                                          ctypes.POINTER(_vp)]
        L.hdg_batch_groups.argtypes = [_vp, _i32p, _i32p, _i32p]
        L.hdg_batch_groups.restype = ctypes.c_int32
        L.hdg_batch_condense.argtypes = [_vp, _vp]
        L.hdg_batch_recover.argtypes = [_vp, _vp]
        L.hdg_batch_step_host_async.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 4 + [_vp]
        L.hdg_batch_autotune.argtypes = [_vp, _i32p, _vp]
        L.hdg_batch_graph_create.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 4
        L.hdg_batch_graph_launch.argtypes = [_vp, _vp]
        L.hdg_batch_launches.argtypes = [_vp]
        L.hdg_batch_launches.restype = ctypes.c_int32
        L.hdg_sys_io.argtypes = [_vp] + [ctypes.POINTER(_vp)] * 4
        L.hdg_sys_workspace_bytes.argtypes = [_vp, ctypes.POINTER(hdg_params)]
        L.hdg_sys_workspace_bytes.restype = ctypes.c_int64
        L.hdg_sys_create_in.argtypes = [_vp, _vp, ctypes.POINTER(hdg_params), _vp, ctypes.c_int64,
                                        ctypes.POINTER(_vp)]
        L.hdg_solver_create.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(_vp)]
        L.hdg_solver_destroy.argtypes = [_vp]
        L.hdg_trace_solve.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double), _vp]
        L.hdg_trace_matvec.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp]
        L.hdg_solver_set_preconditioner.argtypes = [_vp, ctypes.c_int32]
        L.hdg_solver_set_arithmetic.argtypes = [_vp, ctypes.c_int32]
        L.hdg_solver_setup.argtypes = [_vp, _vp]
        L.hdg_solver_precond_apply.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp]
        L.hdg_solver_colors.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.hdg_sys_bucket_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_float)]
        L.hdg_sys_set_source.argtypes = [_vp, _vp]
        L.hdg_solver_create_ws.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int64,
                                           ctypes.POINTER(_vp)]
        L.hdg_solver_workspace_bytes.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
        L.hdg_solver_workspace_bytes.restype = ctypes.c_int64
        L.hdg_solver_create_ws_arith.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                                 ctypes.c_int64, ctypes.POINTER(_vp)]
        L.hdg_solver_create_ws_arith.restype = ctypes.c_int
        L.hdg_solver_workspace_bytes_arith.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.hdg_solver_workspace_bytes_arith.restype = ctypes.c_int64
        L.hdg_solve_step_host.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), _vp]
        L.hdg_trace_solve_ex.argtypes = [_vp, _vp, ctypes.c_int32, _vp, ctypes.c_double, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), _vp]
        L.hdg_adjoint_condense.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.hdg_adapt_indicators.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.hdg_adapt_mark.argtypes = [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp,
                                     ctypes.POINTER(ctypes.c_int32), _vp]
        L.hdg_newton_update.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.hdg_residual_norm.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), _vp]
        L.hdg_sys_set_cfl.argtypes = [_vp, ctypes.c_double]
        L.hdg_autotune.argtypes = [_vp, _vp, _vp, _i32p, _vp]
        L.hdg_cfl_law.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double]
        L.hdg_cfl_law.restype = ctypes.c_double
        _lib = L
    return _lib


def _check(st, ctx_handle=None, what=""):
    if st != HDG_OK:
        msg = lib().hdg_last_error(ctx_handle).decode() if ctx_handle else what
        raise HdgError(st, msg or what)


def _ptr(t) -> int:
    """Device pointer of a contiguous float64/int CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def cfl_law(n: int, c0: float = 1e6, c1: float = 1e3, n0: int = 4, cfl_prev: float = 0.0, res_prev: float = 1.0,
            res_cur: float = 1.0) -> float:
    """hdg_cfl_law: CFL^n of Eq. (cfl) (host only)."""
    return float(lib().hdg_cfl_law(int(n), float(c0), float(c1), int(n0), float(cfl_prev), float(res_prev),
                                   float(res_cur)))


def adapt_mark(ctx: "Context", eta2, sensor, code, theta=0.05, eps_s=1e-6, stream=None) -> int:
    """hdg_adapt_mark: Doerfler marking and h/p choice into the int8 device tensor `code`; returns |M|."""
    nm = ctypes.c_int32()
    _check(lib().hdg_adapt_mark(ctx.h, int(eta2.numel()), _ptr(eta2), _ptr(sensor), float(theta), float(eps_s),
                                _ptr(code), ctypes.byref(nm), _stream(stream)), ctx.h)
    return int(nm.value)


class Solver:
    """hdg_solver_create / hdg_trace_solve / hdg_trace_matvec: GMRES on the trace system of a System."""

    BLOCK_JACOBI, BLOCK_SGS, BLOCK_ILU0, BLOCK_ILU0_F32 = 0, 1, 2, 3

    def __init__(self, system: "System", restart: int = 30, precond: int = 0, workspace=None, arith: int = 0):
        """precond: 0 block Jacobi, 1 multicolor block symmetric Gauss-Seidel, 2 block ILU(0)
        in the multicolor order, 3 the same with binary32 factors.  workspace: optional (device pointer, bytes) holding every
        device buffer (hdg_solver_create_ws_arith; size from ``workspace_bytes`` with the same arith).
        arith: the GMRES arithmetic (0 binary64, 1 float-float; hdg_solver_set_arithmetic)."""
        h = _vp()
        if workspace is None:
            _check(lib().hdg_solver_create(system.h, int(restart), ctypes.byref(h)), system.ctx.h)
            self.h, self.sys = h, system
            _check(lib().hdg_solver_set_preconditioner(h, int(precond)), system.ctx.h)
            if arith:
                self.set_arithmetic(arith)
        else:
            ptr, nbytes = workspace
            _check(lib().hdg_solver_create_ws_arith(system.h, int(restart), int(precond), int(arith),
                                                    ctypes.c_void_p(int(ptr)), int(nbytes), ctypes.byref(h)),
                   system.ctx.h)
            self.h, self.sys = h, system

    @staticmethod
    def workspace_bytes(mesh: "Mesh", restart: int = 30, precond: int = 0, arith: int = 0) -> int:
        """hdg_solver_workspace_bytes_arith: device bytes of a solver on this mesh (for a workspace)."""
        n = int(lib().hdg_solver_workspace_bytes_arith(mesh.h, int(restart), int(precond), int(arith)))
        if n < 0:
            raise HdgError(HDG_EINVAL, "hdg_solver_workspace_bytes: invalid arguments")
        return n

    def step_host(self, U, Lam, dU, dLam, rtol=1e-10, max_iter=3000, stream=None):
        """hdg_solve_step_host: one Newton step from pinned host tensors (blocking);
        returns (iterations, rel. residual)."""
        def hp(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        it, rel = ctypes.c_int32(), ctypes.c_double()
        _check(lib().hdg_solve_step_host(self.sys.h, self.h, hp(U), hp(Lam), hp(dU), hp(dLam), float(rtol),
                                         int(max_iter), ctypes.byref(it), ctypes.byref(rel), _stream(stream)),
               self.sys.ctx.h)
        return int(it.value), float(rel.value)

    def solve(self, dLam, rtol=1e-12, max_iter=500, stream=None, check=True, rhs=None, transpose=False):
        """Solve K dLam = E (or K^T dLam = rhs) in place (dLam holds the initial guess);
        returns (iterations, rel. residual)."""
        it, rel = ctypes.c_int32(), ctypes.c_double()
        st = lib().hdg_trace_solve_ex(self.h, _ptr(rhs) if rhs is not None else None, int(bool(transpose)),
                                      _ptr(dLam), float(rtol), int(max_iter), ctypes.byref(it),
                                      ctypes.byref(rel), _stream(stream))
        if check:
            _check(st, self.sys.ctx.h)
        return int(it.value), float(rel.value)

    def matvec(self, x, y, stream=None, transpose=False):
        """hdg_trace_matvec: y = K x (or K^T x) for device tensors."""
        _check(lib().hdg_trace_matvec(self.h, _ptr(x), _ptr(y), int(bool(transpose)), _stream(stream)),
               self.sys.ctx.h)

    def set_preconditioner(self, kind: int):
        """hdg_solver_set_preconditioner: 0 block Jacobi, 1 block SGS, 2 block ILU(0), 3 ILU(0) binary32."""
        _check(lib().hdg_solver_set_preconditioner(self.h, int(kind)), self.sys.ctx.h)

    BINARY64, FLOAT_FLOAT = 0, 1

    def set_arithmetic(self, arith: int):
        """hdg_solver_set_arithmetic: GMRES products and Krylov updates in binary64 (0) or in
        double-word arithmetic on the binary32 pipe (1)."""
        _check(lib().hdg_solver_set_arithmetic(self.h, int(arith)), self.sys.ctx.h)

    def setup(self, stream=None):
        """Factor the preconditioner for the system's current K (synchronises the stream)."""
        _check(lib().hdg_solver_setup(self.h, _stream(stream)), self.sys.ctx.h)

    def precond_apply(self, r, z, stream=None, transpose=False):
        """z = M^{-1} r (or M^{-T} r) with the factors of the last setup or solve."""
        _check(lib().hdg_solver_precond_apply(self.h, _ptr(r), _ptr(z), int(bool(transpose)), _stream(stream)),
               self.sys.ctx.h)

    def colors(self):
        """(face -> color array, number of colors) of the multicolor order."""
        n = ctypes.c_int32()
        lib().hdg_solver_colors(self.h, None, ctypes.byref(n))
        out = np.empty(self.sys.mesh.n_face, dtype=np.int32)
        _check(lib().hdg_solver_colors(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(n)),
               self.sys.ctx.h)
        return out, int(n.value)

    def close(self):
        if getattr(self, "h", None):
            lib().hdg_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hdg_debug_tables(which: int, p: int, pe: int = 0, lf: int = 0, flip: int = 0) -> np.ndarray:
    """Host-only copy of one of the library's quadrature/basis tables."""
    out = np.zeros(4096)
    n = lib().hdg_debug_tables(which, p, pe, lf, flip, out.ctypes.data_as(_dp), out.size)
    if n < 0:
        raise HdgError(HDG_EINVAL, "no such table")
    return out[:n].copy()


def hdg_condense_noalloc(mesh: "Mesh", params: Params, U, Lam, X, K, E, res_u, res_lam, status, stream=None):
    """Allocation-free condensation into caller device tensors (for callers that
    cannot allocate device memory at call time).  Outputs: X [x_len], K [k_len],
    E [lam_len], res_u [u_len], res_lam [lam_len] float64, status [n_elem] int32.
    Calls that overlap on the GPU share the library's fixed work array and race."""
    P = params.c()
    _check(lib().hdg_condense_noalloc(mesh.h, ctypes.byref(P), _ptr(U), _ptr(Lam), _ptr(X), _ptr(K), _ptr(E),
                                      _ptr(res_u), _ptr(res_lam), _ptr(status), _stream(stream)), mesh.ctx.h)


class _DevView:
    """__cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class Context:
    """hdg_create / hdg_destroy."""

    def __init__(self, device: int = 0):
        h = _vp()
        _check(lib().hdg_create(ctypes.byref(h), int(device)), what=f"hdg_create(device={device}) failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().hdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        """hdg_last_error of this context."""
        return lib().hdg_last_error(self.h).decode()


class Mesh:
    """hdg_mesh_create + hdg_mesh_sizes + hdg_mesh_layout (host arrays in, device plan out)."""

    def __init__(self, ctx: Context, elem_xy, elem_vid, elem_p, nfield: int, elem_bc=None):
        xy = np.ascontiguousarray(elem_xy, dtype=np.float64).reshape(-1)
        vid = np.ascontiguousarray(elem_vid, dtype=np.int32).reshape(-1)
        p = np.ascontiguousarray(elem_p, dtype=np.int8).reshape(-1)
        bc = None if elem_bc is None else np.ascontiguousarray(elem_bc, dtype=np.int8).reshape(-1)
        h = _vp()
        _check(lib().hdg_mesh_create_bc(ctx.h, int(p.size), int(nfield), xy.ctypes.data_as(_dp),
                                        vid.ctypes.data_as(_i32p), p.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                        bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if bc is not None else None,
                                        ctypes.byref(h)), ctx.h)
        self.h, self.ctx, self.nfield = h, ctx, nfield
        s = np.zeros(7, np.int64)
        lib().hdg_mesh_sizes(h, s.ctypes.data_as(_i64p))
        self.n_elem, self.n_face, self.u_len, self.lam_len, self.x_len, self.k_len, self.max_nt = (int(v) for v in s)
        nf, ne = self.n_face, self.n_elem
        self.face_vid = np.zeros((nf, 2), np.int32)
        self.face_el = np.zeros((nf, 2), np.int32)
        self.face_p = np.zeros(nf, np.int32)
        self.elem_face = np.zeros((ne, 3), np.int32)
        self.u_off = np.zeros(ne + 1, np.int64)
        self.lam_off = np.zeros(nf + 1, np.int64)
        self.x_off = np.zeros(ne + 1, np.int64)
        self.k_col = np.zeros((nf, 5), np.int32)
        self.k_blkoff = np.zeros(5 * nf + 1, np.int64)
        lib().hdg_mesh_layout(h, self.face_vid.ctypes.data_as(_i32p), self.face_el.ctypes.data_as(_i32p),
                              self.face_p.ctypes.data_as(_i32p), self.elem_face.ctypes.data_as(_i32p),
                              self.u_off.ctypes.data_as(_i64p), self.lam_off.ctypes.data_as(_i64p),
                              self.x_off.ctypes.data_as(_i64p), self.k_col.ctypes.data_as(_i32p),
                              self.k_blkoff.ctypes.data_as(_i64p))
        self.elem_p = p.astype(np.int32)

    def footprint_bytes(self, params: Params) -> int:
        """hdg_footprint_bytes: device bytes a system on this mesh holds (admission)."""
        P = params.c()
        return int(lib().hdg_footprint_bytes(self.h, ctypes.byref(P)))

    def workspace_bytes(self, params: Params) -> int:
        """hdg_sys_workspace_bytes: bytes of caller workspace for hdg_sys_create_in."""
        P = params.c()
        return int(lib().hdg_sys_workspace_bytes(self.h, ctypes.byref(P)))

    def close(self):
        if getattr(self, "h", None):
            lib().hdg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """hdg_sys_create (or hdg_sys_create_in with a device workspace) / hdg_condense /
    hdg_recover / hdg_step_host / hdg_sys_get."""

    def __init__(self, ctx: Context, mesh: Mesh, params: Params, workspace=None):
        P = params.c()
        h = _vp()
        if workspace is None:
            _check(lib().hdg_sys_create(ctx.h, mesh.h, ctypes.byref(P), ctypes.byref(h)), ctx.h)
        else:
            ptr, nbytes = workspace
            _check(lib().hdg_sys_create_in(ctx.h, mesh.h, ctypes.byref(P), int(ptr), int(nbytes), ctypes.byref(h)),
                   ctx.h)
        self.h, self.ctx, self.mesh, self.params = h, ctx, mesh, params
        ptrs = [_vp() for _ in range(6)]
        lib().hdg_sys_get(h, *[ctypes.byref(p) for p in ptrs])
        self._ptrs = [p.value for p in ptrs]

    def condense(self, U, Lam, stream=None):
        """hdg_condense on device tensors U [u_len], Lam [lam_len] (float64)."""
        _check(lib().hdg_condense(self.h, _ptr(U), _ptr(Lam), _stream(stream)), self.ctx.h)

    def recover(self, dLam, dU, stream=None):
        """hdg_recover: dU [u_len] <- X_F - X_B dLam, device tensors."""
        _check(lib().hdg_recover(self.h, _ptr(dLam), _ptr(dU), _stream(stream)), self.ctx.h)

    def step_host(self, U, Lam, dLam, dU, stream=None):
        """hdg_step_host on host (preferably pinned) float64 torch tensors or numpy arrays."""
        def hp(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        _check(lib().hdg_step_host(self.h, hp(U), hp(Lam), hp(dLam), hp(dU), _stream(stream)), self.ctx.h)

    def step_host_async(self, U, Lam, dLam, dU, stream=None):
        """hdg_step_host_async: enqueue the whole step on `stream` from pinned host tensors."""
        def hp(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        _check(lib().hdg_step_host_async(self.h, hp(U), hp(Lam), hp(dLam), hp(dU), _stream(stream)), self.ctx.h)

    def graph_create(self, U, Lam, dLam, dU):
        """hdg_graph_create: capture the whole step for these device tensors."""
        _check(lib().hdg_graph_create(self.h, _ptr(U), _ptr(Lam), _ptr(dLam), _ptr(dU)), self.ctx.h)

    def graph_launch(self, stream=None):
        """hdg_graph_launch: replay the captured step on `stream`."""
        _check(lib().hdg_graph_launch(self.h, _stream(stream)), self.ctx.h)

    @property
    def launches(self) -> int:
        """hdg_sys_launches: kernel launches of the last condense + recover."""
        return int(lib().hdg_sys_launches(self.h))

    def set_source(self, S=None):
        """hdg_sys_set_source: source coefficients (device tensor in U's layout, kept alive
        by this object) or None."""
        self._src = S
        _check(lib().hdg_sys_set_source(self.h, _ptr(S) if S is not None else None), self.ctx.h)

    def bucket_times(self) -> dict:
        """hdg_sys_bucket_times: {p: ms} of each degree bucket in the last multi-bucket condensation."""
        ms = (ctypes.c_float * 5)()
        _check(lib().hdg_sys_bucket_times(self.h, ms), self.ctx.h)
        return {p: float(ms[p]) for p in range(1, 5) if ms[p] >= 0.0}

    def newton_update(self, U, Lam, dU, dLam, stream=None):
        """hdg_newton_update: U += dU, Lam += dLam on device tensors."""
        _check(lib().hdg_newton_update(self.h, _ptr(U), _ptr(Lam), _ptr(dU), _ptr(dLam), _stream(stream)),
               self.ctx.h)

    def residual_norm(self, stream=None) -> float:
        """hdg_residual_norm: ||[N_q; N_w; N_lambda]||_2 of the last condensed state."""
        out = ctypes.c_double()
        _check(lib().hdg_residual_norm(self.h, ctypes.byref(out), _stream(stream)), self.ctx.h)
        return out.value

    def autotune(self, U, Lam, stream=None) -> dict:
        """hdg_autotune: pick the fastest launch shape per degree bucket; returns {p: shape}."""
        out = (ctypes.c_int32 * 5)()
        _check(lib().hdg_autotune(self.h, _ptr(U), _ptr(Lam), out, _stream(stream)), self.ctx.h)
        return {p: int(out[p]) for p in range(1, 5) if out[p] >= 0}

    def adjoint_condense(self, primal: "System", U, Lam, Ftilde, stream=None):
        """hdg_adjoint_condense: adjoint local solves into this system's X, E~ into its E."""
        _check(lib().hdg_adjoint_condense(self.h, primal.h, _ptr(U), _ptr(Lam), _ptr(Ftilde), _stream(stream)),
               self.ctx.h)

    def adapt_indicators(self, U, Uadj, eta2, sensor, stream=None):
        """hdg_adapt_indicators: eta_K^2 (needs Uadj) and the smoothness sensor S_K per element."""
        _check(lib().hdg_adapt_indicators(self.h, _ptr(U), _ptr(Uadj) if Uadj is not None else None,
                                          _ptr(eta2) if eta2 is not None else None,
                                          _ptr(sensor) if sensor is not None else None, _stream(stream)), self.ctx.h)

    def set_cfl(self, cfl: float):
        """hdg_sys_set_cfl: pseudo-time CFL number of the following condensations."""
        _check(lib().hdg_sys_set_cfl(self.h, float(cfl)), self.ctx.h)
        self.params.cfl = float(cfl)

    def io_views(self):
        """hdg_sys_io: zero-copy torch views of the system's device staging buffers U, Lam, dLam, dU
        (the inputs and output of the batched calls)."""
        import torch
        ptrs = [_vp() for _ in range(4)]
        _check(lib().hdg_sys_io(self.h, *[ctypes.byref(p) for p in ptrs]), self.ctx.h)
        m = self.mesh
        n = [m.u_len, m.lam_len, m.lam_len, m.u_len]
        return {nm: torch.as_tensor(_DevView(p.value, k, "<f8"), device=f"cuda:{self.ctx.device}")
                for nm, p, k in zip(["U", "Lam", "dLam", "dU"], ptrs, n)}

    def views(self):
        """Zero-copy torch views of X, K, E, res_u, res_lam, elem_status."""
        import torch
        m = self.mesh
        n = [m.x_len, m.k_len, m.lam_len, m.u_len, m.lam_len, m.n_elem]
        ty = ["<f8"] * 5 + ["<i4"]
        names = ["X", "K", "E", "res_u", "res_lam", "status"]
        return {nm: torch.as_tensor(_DevView(p, k, t), device=f"cuda:{self.ctx.device}")
                for nm, p, k, t in zip(names, self._ptrs, n, ty)}

    def close(self):
        if getattr(self, "h", None):
            lib().hdg_sys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptrs(arrs):
    """ctypes array of the host addresses of torch tensors or numpy arrays."""
    out = (_vp * len(arrs))()
    for i, a in enumerate(arrs):
        out[i] = a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    return out


class Batch:
    """hdg_batch_*: one condensation launch per (model, degree) group over the elements of several
    systems; each system's results are bitwise those of condensing it alone."""

    def __init__(self, ctx: Context, systems: list, workspace=None, stream=None):
        """workspace=(device pointer, bytes): hdg_batch_create_in (work list uploaded on `stream`)."""
        arr = (_vp * len(systems))(*[s.h for s in systems])
        h = _vp()
        if workspace is None:
            _check(lib().hdg_batch_create(ctx.h, len(systems), arr, ctypes.byref(h)), ctx.h)
        else:
            ptr, nbytes = workspace
            _check(lib().hdg_batch_create_in(ctx.h, len(systems), arr, int(ptr), int(nbytes), _stream(stream),
                                             ctypes.byref(h)), ctx.h)
        self.h, self.ctx, self.systems = h, ctx, list(systems)

    @staticmethod
    def workspace_bytes(systems: list) -> int:
        """hdg_batch_workspace_bytes: device bytes of the work list of a batch of these systems."""
        arr = (_vp * len(systems))(*[s.h for s in systems])
        return int(lib().hdg_batch_workspace_bytes(len(systems), arr))

    def groups(self) -> list:
        """[(model, p, n_items)] of the batch's launches."""
        m, p, n = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)()
        g = int(lib().hdg_batch_groups(self.h, m, p, n))
        return [(int(m[i]), int(p[i]), int(n[i])) for i in range(g)]

    def condense(self, stream=None):
        _check(lib().hdg_batch_condense(self.h, _stream(stream)), self.ctx.h)

    def recover(self, stream=None):
        _check(lib().hdg_batch_recover(self.h, _stream(stream)), self.ctx.h)

    def step_host_async(self, U, Lam, dLam, dU, stream=None):
        """Lists (one per system) of pinned host tensors."""
        self._keep = (_host_ptrs(U), _host_ptrs(Lam), _host_ptrs(dLam), _host_ptrs(dU))
        _check(lib().hdg_batch_step_host_async(self.h, *self._keep, _stream(stream)), self.ctx.h)

    def autotune(self, stream=None) -> dict:
        out = (ctypes.c_int32 * 10)()
        _check(lib().hdg_batch_autotune(self.h, out, _stream(stream)), self.ctx.h)
        return {(md, p): int(out[md * 5 + p]) for md in range(2) for p in range(1, 5) if out[md * 5 + p] >= 0}

    def graph_create(self, U, Lam, dLam, dU):
        self._gkeep = (_host_ptrs(U), _host_ptrs(Lam), _host_ptrs(dLam), _host_ptrs(dU))
        _check(lib().hdg_batch_graph_create(self.h, *self._gkeep), self.ctx.h)

    def graph_launch(self, stream=None):
        _check(lib().hdg_batch_graph_launch(self.h, _stream(stream)), self.ctx.h)

    @property
    def launches(self) -> int:
        return int(lib().hdg_batch_launches(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().hdg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
