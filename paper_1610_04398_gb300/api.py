"""Thin Python binding of the C ABI in ``include/pp.h`` (ctypes).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``libpp.so``.  Device arrays are torch CUDA tensors (their ``data_ptr``); calls
are ordered on torch's current CUDA stream at the time of the call.  There is no
CPU fallback: if ``libpp.so`` cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PP_OK, PP_ERR_ARG, PP_ERR_STATE, PP_ERR_OOM, PP_ERR_CUDA, PP_ERR_TIMEOUT, PP_ERR_BUDGET = range(7)
PP_FP64, PP_MIXED = 0, 1
PP_NEAREST, PP_BILINEAR = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpp.so")
_LOCK = threading.Lock()
_LIB = None


class PPError(RuntimeError):
    """A pp_* call returned a non-zero pp_status."""

    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {error_string(status)} (status {status})")


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("precision", ctypes.c_int), ("lift", ctypes.c_double),
                ("interp", ctypes.c_int), ("uinf_x", ctypes.c_double), ("uinf_y", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("tile", ctypes.c_int), ("theta_surface", ctypes.c_double),
                ("m2l_tensor", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("order", ctypes.c_int), ("theta", ctypes.c_double), ("tile", ctypes.c_int),
                ("theta_surface", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("grid", _Grid), ("h", ctypes.c_double), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("chi", ctypes.c_void_p), ("us_x", ctypes.c_void_p), ("us_y", ctypes.c_void_p),
                ("lam", ctypes.c_double), ("nu", ctypes.c_double), ("rho", ctypes.c_double),
                ("lift", ctypes.c_double), ("interp", ctypes.c_int), ("uinf_x", ctypes.c_double),
                ("uinf_y", ctypes.c_double), ("npts", ctypes.c_int), ("points", ctypes.c_void_p),
                ("normals", ctypes.c_void_p), ("dS", ctypes.c_void_p), ("p_out", ctypes.c_void_p),
                ("per_point", ctypes.c_void_p), ("forces", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("queued", "running", "completed", "failed", "plans_resident",
                                              "plans_created", "plans_evicted", "bytes_held")]


PP_SERVER_QUEUED, PP_SERVER_RUNNING, PP_SERVER_DONE, PP_SERVER_FAILED, PP_SERVER_CANCELLED = range(5)


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("order", ctypes.c_int), ("levels", ctypes.c_int),
                ("precision", ctypes.c_int), ("h", ctypes.c_double), ("theta", ctypes.c_double),
                ("n_near", ctypes.c_int), ("n_m2l", ctypes.c_int * 4), ("near_pairs", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("m2l_pairs_leaf", ctypes.c_int64),
                ("theta_surface", ctypes.c_double), ("near_kernel", ctypes.c_int), ("downward", ctypes.c_int)]


def load(path: str = None):
    """Load libpp.so and declare every exported signature (raises if missing)."""
    global _LIB
    with _LOCK:
        if _LIB is not None and path is None:
            return _LIB
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libpp.so not found at {p}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        sig = {
            "pp_options_default": (None, [ctypes.POINTER(_Options)]),
            "pp_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), _Grid, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_double, ctypes.POINTER(_Options)]),
            "pp_plan_destroy": (ctypes.c_int, [vp]),
            "pp_plan_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Options),
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
            "pp_plan_set_stream": (ctypes.c_int, [vp, vp]),
            "pp_rhs": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_double, vp]),
            "pp_pressure_solve": (ctypes.c_int, [vp, vp]),
            "pp_pressure_solve_fft": (ctypes.c_int, [vp, vp]),
            "pp_atree_create": (ctypes.c_int, [ctypes.c_int, ip, ip, ip, ctypes.c_double, ctypes.POINTER(vp)]),
            "pp_atree_create_device": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, ctypes.c_double, vp,
                                                      ctypes.POINTER(vp)]),
            "pp_atree_sizes": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
            "pp_atree_boxes": (ctypes.c_int, [vp, ip, ip, ip, ip, ip, ip]),
            "pp_atree_lists": (ctypes.c_int, [vp, ip, ip]),
            "pp_atree_destroy": (ctypes.c_int, [vp]),
            "pp_atree_solve": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp]),
            "pp_atree_surface_pressure": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, ctypes.c_double, vp, vp]),
            "pp_surface_traction": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp, vp, ctypes.c_double,
                                                   vp, vp]),
            "pp_plan_info": (ctypes.c_int, [vp, ctypes.POINTER(PlanInfo)]),
            "pp_plan_device_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
            "pp_get_expansion": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp]),
            "pp_near_offsets": (ctypes.c_int, [ctypes.c_double, ip, ctypes.c_int]),
            "pp_m2l_offsets": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ip, ctypes.c_int]),
            "pp_m2l_entries": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ip, ctypes.c_int]),
            "pp_error_string": (ctypes.c_char_p, [ctypes.c_int]),
            "pp_surface_forces_noalloc": (ctypes.c_int, [ctypes.c_int, _Grid, ctypes.c_double, vp, vp,
                                                         ctypes.c_int, vp, vp, vp, vp, ctypes.c_double,
                                                         ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                         ctypes.c_double, ctypes.c_double, vp, vp, vp]),
            "pp_step_graph_create": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, ctypes.c_int,
                                                    vp, vp, vp, ctypes.c_double, vp, vp, ctypes.POINTER(vp)]),
            "pp_step_graph_launch": (ctypes.c_int, [vp, vp]),
            "pp_step_graph_destroy": (ctypes.c_int, [vp]),
            "pp_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
            "pp_batch_launch": (ctypes.c_int, [vp, vp]),
            "pp_batch_destroy": (ctypes.c_int, [vp]),
            "pp_server_config_default": (None, [ctypes.POINTER(ServerConfig)]),
            "pp_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
            "pp_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
            "pp_server_cancel": (ctypes.c_int, [vp, ctypes.c_int64]),
            "pp_server_query": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
            "pp_server_wait": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_double]),
            "pp_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
            "pp_server_destroy": (ctypes.c_int, [vp]),
            "pp_pipeline_create": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int, vp, ctypes.c_double,
                                                  ctypes.POINTER(vp)]),
            "pp_pipeline_submit": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "pp_pipeline_wait": (ctypes.c_int, [vp]),
            "pp_pipeline_destroy": (ctypes.c_int, [vp]),
            "pp_penal_force": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, ctypes.c_double, vp]),
            "pp_body_moments": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "pp_plan_enable_timing": (ctypes.c_int, [vp, ctypes.c_int]),
            "pp_measure_alu_peaks": (ctypes.c_int, [dp, ctypes.c_int, vp]),
            "pp_plan_stage_times": (ctypes.c_int, [vp, dp, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _LIB = lib
        return lib


def error_string(status: int) -> str:
    try:
        return load().pp_error_string(int(status)).decode()
    except Exception:  # library missing: still say something useful
        return f"status {status}"


def _check(fn: str, st: int):
    if st != PP_OK:
        raise PPError(fn, st)


def _hptr(t, dtype, numel: int = None, name: str = "array"):
    """Host pointer of a contiguous CPU tensor of the given dtype (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU tensor (page-locked for overlapped copies)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, dtype, numel: int = None, name: str = "array"):
    """Device pointer of a contiguous CUDA tensor of the given dtype (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def pp_near_offsets(theta: float) -> np.ndarray:
    """Same-level leaf offsets in the near field at acceptance parameter theta (host only)."""
    lib = load()
    n = lib.pp_near_offsets(float(theta), None, 0)
    if n < 0:
        raise PPError("pp_near_offsets", -n)
    buf = (ctypes.c_int * (2 * n))()
    lib.pp_near_offsets(float(theta), buf, n)
    return np.array(buf, dtype=np.int64).reshape(n, 2)


def pp_m2l_offsets(theta: float, child: int) -> np.ndarray:
    """Multipole-to-local offsets of a box at child position ``child`` (host only)."""
    lib = load()
    n = lib.pp_m2l_offsets(float(theta), int(child), None, 0)
    if n < 0:
        raise PPError("pp_m2l_offsets", -n)
    buf = (ctypes.c_int * (2 * n))()
    lib.pp_m2l_offsets(float(theta), int(child), buf, n)
    return np.array(buf, dtype=np.int64).reshape(n, 2)


def pp_m2l_entries(theta: float, child: int) -> np.ndarray:
    """Interaction-list entries (dx, dy, kind) of a box at child position ``child``:
    kind 0 same-level source, kind 1 parent-level source (host only)."""
    lib = load()
    n = lib.pp_m2l_entries(float(theta), int(child), None, 0)
    if n < 0:
        raise PPError("pp_m2l_entries", -n)
    buf = (ctypes.c_int * (3 * n))()
    lib.pp_m2l_entries(float(theta), int(child), buf, n)
    return np.array(buf, dtype=np.int64).reshape(n, 3)


def plan_bytes(n: int, order: int = 20, theta: float = 0.5, *, precision: str = "fp64", tile: int = 16,
               npts: int = 0, m2l_tensor: bool = False) -> int:
    """pp_plan_bytes: device bytes a plan with these settings holds, its surface scratch grown
    for calls of up to ``npts`` points (host only, allocates nothing)."""
    lib = load()
    opt = _Options()
    lib.pp_options_default(ctypes.byref(opt))
    opt.precision = {"fp64": PP_FP64, "mixed": PP_MIXED}[precision]
    opt.tile = int(tile)
    opt.m2l_tensor = int(bool(m2l_tensor))
    out = ctypes.c_int64()
    _check("pp_plan_bytes", lib.pp_plan_bytes(int(n), int(order), float(theta), ctypes.byref(opt), int(npts),
                                              ctypes.byref(out)))
    return out.value


def measure_alu_peaks(reps: int = 5) -> dict:
    """pp_measure_alu_peaks on the current device and torch's current stream."""
    lib = load()
    out = (ctypes.c_double * 7)()
    _check("pp_measure_alu_peaks", lib.pp_measure_alu_peaks(out, int(reps), _stream_ptr()))
    return {"fp32_tflops": out[0], "lg2_gops": out[1], "fp64_tflops": out[2],
            "ms": {"fp32_fma": out[3], "lg2": out[4], "fp64_fma": out[5]}, "sms": int(out[6])}


class Plan:
    """A pp_plan: fixed grid, order and theta; owns the device workspace.

    ``precision`` is "fp64" (grid arrays float64) or "mixed" (grid arrays float32).
    ``m2l_tensor``: mixed plans of order 12 with theta >= 0.5 run the multipole-to-local
    translations on the tensor cores (``info().downward == 3``); other plans keep the FP32-core
    kernel.
    """

    def __init__(self, n: int, h: float, order: int = 20, theta: float = 0.5, *, x0: float = 0.0,
                 y0: float = 0.0, rho: float = 1.0, precision: str = "fp64", lift: float = None,
                 interp: str = "nearest", uinf=(1.0, 0.0), tile: int = 16, theta_surface: float = 0.0,
                 m2l_tensor: bool = False):
        import torch
        lib = load()
        opt = _Options()
        lib.pp_options_default(ctypes.byref(opt))
        opt.rho = float(rho)
        opt.precision = {"fp64": PP_FP64, "mixed": PP_MIXED}[precision]
        opt.lift = -1.0 if lift is None else float(lift)
        opt.interp = {"nearest": PP_NEAREST, "bilinear": PP_BILINEAR}[interp]
        opt.uinf_x, opt.uinf_y = float(uinf[0]), float(uinf[1])
        opt.stream = _stream_ptr()
        opt.tile = int(tile)
        opt.theta_surface = float(theta_surface)
        opt.m2l_tensor = int(bool(m2l_tensor))
        self._lib = lib
        self._h = ctypes.c_void_p()
        self.n = int(n)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        _check("pp_plan_create", lib.pp_plan_create(ctypes.byref(self._h), _Grid(int(n), float(x0), float(y0)),
                                                    float(h), int(order), float(theta), ctypes.byref(opt)))

    # -- lifecycle ---------------------------------------------------------------
    def destroy(self):
        if self._h and self._h.value:
            self._lib.pp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def _sync_stream(self):
        _check("pp_plan_set_stream", self._lib.pp_plan_set_stream(self._h, _stream_ptr()))

    # -- the path ------------------------------------------------------------------
    def rhs(self, u, v, chi, usx, usy, lam: float, f_out=None):
        """pp_rhs: Poisson source and leaf multipoles (fields n*n, plan dtype)."""
        nn = self.n * self.n
        self._sync_stream()
        args = [_dptr(a, self.dtype, nn, nm) for a, nm in ((u, "u"), (v, "v"), (chi, "chi"),
                                                            (usx, "us_x"), (usy, "us_y"))]
        _check("pp_rhs", self._lib.pp_rhs(self._h, *args, float(lam), _dptr(f_out, self.dtype, nn, "f_out")))

    def pressure_solve(self, p_out=None):
        """pp_pressure_solve: pressure at every cell into p_out (n*n, plan dtype) or NULL."""
        self._sync_stream()
        _check("pp_pressure_solve",
               self._lib.pp_pressure_solve(self._h, _dptr(p_out, self.dtype, self.n * self.n, "p_out")))

    def pressure_solve_fft(self, p_out):
        """pp_pressure_solve_fft: the same discrete sum at every cell by the zero-padded FFT
        convolution (Hockney) into p_out (n*n, plan dtype).  The first call forms the
        transformed kernel and synchronises the plan's stream."""
        self._sync_stream()
        _check("pp_pressure_solve_fft",
               self._lib.pp_pressure_solve_fft(self._h, _dptr(p_out, self.dtype, self.n * self.n, "p_out")))

    def surface_traction(self, u, v, points, normals, nu: float, dS=None, per_point=None, forces=None):
        """pp_surface_traction. points/normals: (npts, 2) float64 CUDA tensors.

        ``forces``: None (returned as a host numpy array, stream synchronised), or a
        6-element float64 CUDA tensor written stream-ordered (returns None)."""
        import torch
        npts = int(points.shape[0])
        nn = self.n * self.n
        self._sync_stream()
        host = None
        if forces is None:
            host = np.zeros(6, np.float64)
            fptr = ctypes.c_void_p(host.ctypes.data)
        else:
            fptr = _dptr(forces, torch.float64, 6, "forces")
        st = self._lib.pp_surface_traction(
            self._h, _dptr(u, self.dtype, nn, "u"), _dptr(v, self.dtype, nn, "v"), npts,
            _dptr(points, torch.float64, 2 * npts, "points"), _dptr(normals, torch.float64, 2 * npts, "normals"),
            _dptr(dS, torch.float64, npts, "dS"), float(nu), _dptr(per_point, torch.float64, 5 * npts, "per_point"),
            fptr)
        _check("pp_surface_traction", st)
        return host

    def penal_force(self, u, v, chi, usx, usy, lam: float, forces=None):
        """pp_penal_force (Eq. dragPenal): [Fx, Fy, drag, lift].  With ``forces`` (a CUDA
        float64 tensor of 4) the result stays on the device; otherwise a numpy array."""
        import torch
        nn = self.n * self.n
        args = [_dptr(a, self.dtype, nn, nm) for a, nm in ((u, "u"), (v, "v"), (chi, "chi"),
                                                            (usx, "us_x"), (usy, "us_y"))]
        if forces is not None:
            _check("pp_penal_force", self._lib.pp_penal_force(self._h, *args, float(lam),
                                                              _dptr(forces, torch.float64, 4, "forces")))
            return forces
        host = np.zeros(4)
        _check("pp_penal_force", self._lib.pp_penal_force(
            self._h, *args, float(lam), host.ctypes.data_as(ctypes.c_void_p)))
        return host

    def body_moments(self, u, v, chi, out=None):
        """pp_body_moments: [M, u_CM_x, u_CM_y] of the body marked by chi (Sec. 3.3).  With
        ``out`` (a CUDA float64 tensor of 3) the result stays on the device; otherwise numpy."""
        import torch
        nn = self.n * self.n
        args = [_dptr(a, self.dtype, nn, nm) for a, nm in ((u, "u"), (v, "v"), (chi, "chi"))]
        self._sync_stream()
        if out is not None:
            _check("pp_body_moments", self._lib.pp_body_moments(self._h, *args, _dptr(out, torch.float64, 3, "out")))
            return out
        host = np.zeros(3)
        _check("pp_body_moments", self._lib.pp_body_moments(self._h, *args, host.ctypes.data_as(ctypes.c_void_p)))
        return host

    def capture_step(self, u, v, chi, usx, usy, lam: float, p_out=None, points=None, normals=None,
                     nu: float = 0.0, dS=None, per_point=None, forces=None) -> "StepGraph":
        """pp_step_graph_create: the whole step (source, solve, surface) as one CUDA graph."""
        import torch
        nn = self.n * self.n
        npts = 0 if points is None else int(points.shape[0])
        g = ctypes.c_void_p()
        args = [_dptr(a, self.dtype, nn, nm) for a, nm in ((u, "u"), (v, "v"), (chi, "chi"),
                                                            (usx, "us_x"), (usy, "us_y"))]
        st = self._lib.pp_step_graph_create(
            self._h, *args, float(lam), _dptr(p_out, self.dtype, nn, "p_out"), npts,
            _dptr(points, torch.float64, 2 * npts, "points"), _dptr(normals, torch.float64, 2 * npts, "normals"),
            _dptr(dS, torch.float64, npts, "dS"), float(nu), _dptr(per_point, torch.float64, 5 * npts, "per_point"),
            _dptr(forces, torch.float64, 6, "forces"), ctypes.byref(g))
        _check("pp_step_graph_create", st)
        return StepGraph(self, g)

    STAGES = ("rhs_p2m", "upward", "downward", "leaf", "leaf_m2l", "surface")

    def enable_timing(self, on: bool = True):
        """Record CUDA events around each stage on the plan's stream."""
        _check("pp_plan_enable_timing", self._lib.pp_plan_enable_timing(self._h, int(bool(on))))

    def stage_times(self) -> dict:
        """Latest duration (ms) of each stage, -1 for a stage that has not run."""
        buf = (ctypes.c_double * len(self.STAGES))()
        st = self._lib.pp_plan_stage_times(self._h, buf, len(self.STAGES))
        if st < 0:
            raise PPError("pp_plan_stage_times", -st)
        return {name: buf[i] for i, name in enumerate(self.STAGES)}

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check("pp_plan_info", self._lib.pp_plan_info(self._h, ctypes.byref(inf)))
        return inf

    def device_status(self):
        """pp_plan_device_status: the four device flags (cleared on read); raises PPError
        (PP_ERR_TIMEOUT) if a tensor-core kernel's bounded wait gave up."""
        buf = (ctypes.c_int * 4)()
        st = self._lib.pp_plan_device_status(self._h, buf)
        flags = [buf[i] for i in range(4)]
        if st != PP_OK:
            raise PPError("pp_plan_device_status", st)
        return flags

    def get_expansion(self, kind: str, level: int):
        """Scaled coefficients of one level as a complex128 CUDA tensor [4^level, order+1]."""
        import torch
        inf = self.info()
        nb = 4 ** int(level)
        out = torch.empty(nb * inf.order * 2 + nb * 2, dtype=torch.float64, device="cuda")
        self._sync_stream()
        _check("pp_get_expansion", self._lib.pp_get_expansion(
            self._h, {"multipole": 0, "local": 1}[kind], int(level), ctypes.c_void_p(out.data_ptr())))
        return torch.view_as_complex(out.view(nb, inf.order + 1, 2))


def accelerations(forces, moments, dt: float):
    """The deforming body's acceleration over a sequence of snapshots dt apart (Sec. 3.3):
    Eq. aSF, a_SF^n = (F_P^n + F_nu^n) / M^n, and Eq. aPenal, a_penal^n = (u_CM^(n+1) -
    u_CM^(n-1)) / (2 dt), for the interior snapshots n = 1 .. N-2.  ``forces``: N rows of
    pp_surface_traction's 6 forces; ``moments``: N rows of pp_body_moments.  Host arithmetic
    on the results of those two calls.  Returns (a_SF, a_penal), each (N-2, 2)."""
    F = np.asarray(forces, np.float64)
    m = np.asarray(moments, np.float64)
    a_sf = np.stack([F[1:-1, 0] + F[1:-1, 2], F[1:-1, 1] + F[1:-1, 3]], axis=1) / m[1:-1, 0:1]
    a_pen = (m[2:, 1:3] - m[:-2, 1:3]) / (2.0 * dt)
    return a_sf, a_pen


class StepGraph:
    """A captured step (pp_graph); launch() replays it on torch's current stream."""

    def __init__(self, plan: Plan, handle):
        self.plan = plan  # keeps the plan alive while the graph exists
        self._h = handle

    def launch(self):
        _check("pp_step_graph_launch", self.plan._lib.pp_step_graph_launch(self._h, _stream_ptr()))

    def destroy(self):
        if self._h and self._h.value:
            self.plan._lib.pp_step_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Pipeline:
    """pp_pipeline: snapshots streamed from host memory; uploads, solves and downloads
    of neighbouring snapshots overlap.  Host tensors should be pinned (``pin_memory()``)
    and must stay alive and unmodified until ``wait()`` returns."""

    def __init__(self, plan: Plan, lam: float, npts: int = 0, dS=None, nu: float = 0.0):
        import torch
        self.plan = plan
        self.npts = int(npts)
        self._keep = [dS]
        self._h = ctypes.c_void_p()
        _check("pp_pipeline_create", plan._lib.pp_pipeline_create(
            plan._h, float(lam), self.npts, _dptr(dS, torch.float64, self.npts, "dS"), float(nu),
            ctypes.byref(self._h)))

    def submit(self, u, v, chi, usx, usy, points=None, normals=None, p_out=None, forces=None):
        import torch
        nn = self.plan.n * self.plan.n
        dt = self.plan.dtype
        args = [_hptr(a, dt, nn, nm) for a, nm in ((u, "u"), (v, "v"), (chi, "chi"), (usx, "us_x"),
                                                    (usy, "us_y"))]
        st = self.plan._lib.pp_pipeline_submit(
            self._h, *args, _hptr(points, torch.float64, 2 * self.npts, "points"),
            _hptr(normals, torch.float64, 2 * self.npts, "normals"), _hptr(p_out, dt, nn, "p_out"),
            _hptr(forces, torch.float64, 6, "forces"))
        _check("pp_pipeline_submit", st)

    def wait(self):
        _check("pp_pipeline_wait", self.plan._lib.pp_pipeline_wait(self._h))

    def destroy(self):
        if self._h and self._h.value:
            self.plan._lib.pp_pipeline_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """pp_batch: several step graphs (independent snapshots, any grid sizes) launched as
    one CUDA graph whose branches run concurrently."""

    def __init__(self, graphs):
        self.graphs = list(graphs)  # keep plans, buffers and graphs alive
        lib = load()
        arr = (ctypes.c_void_p * len(self.graphs))(*[g._h.value for g in self.graphs])
        self._h = ctypes.c_void_p()
        self._lib = lib
        _check("pp_batch_create", lib.pp_batch_create(len(self.graphs), arr, ctypes.byref(self._h)))

    def launch(self):
        _check("pp_batch_launch", self._lib.pp_batch_launch(self._h, _stream_ptr()))

    def destroy(self):
        if self._h and self._h.value:
            self._lib.pp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Server:
    """pp_server: continuous-batching solve loop with HBM-budget admission.

    ``submit`` takes torch CUDA tensors of the server's precision (they must stay alive
    until the request is finished; the Python object keeps references until then)."""

    def __init__(self, budget_bytes: int = 8 << 30, slots: int = 8, precision: str = "mixed",
                 order: int = 12, theta: float = 0.6, tile: int = 16, theta_surface: float = 0.0):
        import torch
        self._lib = load()
        cfg = ServerConfig()
        self._lib.pp_server_config_default(ctypes.byref(cfg))
        cfg.budget_bytes, cfg.slots = int(budget_bytes), int(slots)
        cfg.precision = {"fp64": PP_FP64, "mixed": PP_MIXED}[precision]
        cfg.order, cfg.theta, cfg.tile = int(order), float(theta), int(tile)
        cfg.theta_surface = float(theta_surface)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self._h = ctypes.c_void_p()
        self._keep = {}
        _check("pp_server_create", self._lib.pp_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))

    def submit(self, n, h, u, v, chi, usx, usy, lam, *, x0=0.0, y0=0.0, nu=0.0, rho=1.0, lift=None,
               interp="nearest", uinf=(1.0, 0.0), points=None, normals=None, dS=None, p_out=None,
               per_point=None, forces=None) -> int:
        import torch
        nn = int(n) * int(n)
        npts = 0 if points is None else int(points.shape[0])
        r = Request()
        r.grid = _Grid(int(n), float(x0), float(y0))
        r.h = float(h)
        r.u, r.v, r.chi, r.us_x, r.us_y = [_dptr(a, self.dtype, nn, nm) for a, nm in
                                           ((u, "u"), (v, "v"), (chi, "chi"), (usx, "us_x"), (usy, "us_y"))]
        r.lam, r.nu, r.rho = float(lam), float(nu), float(rho)
        r.lift = -1.0 if lift is None else float(lift)
        r.interp = {"nearest": PP_NEAREST, "bilinear": PP_BILINEAR}[interp]
        r.uinf_x, r.uinf_y = float(uinf[0]), float(uinf[1])
        r.npts = npts
        r.points = _dptr(points, torch.float64, 2 * npts, "points")
        r.normals = _dptr(normals, torch.float64, 2 * npts, "normals")
        r.dS = _dptr(dS, torch.float64, npts, "dS")
        r.p_out = _dptr(p_out, self.dtype, nn, "p_out")
        r.per_point = _dptr(per_point, torch.float64, 5 * npts, "per_point")
        r.forces = _dptr(forces, torch.float64, 6, "forces")
        rid = ctypes.c_int64()
        # the server's streams must see the inputs written on torch's current stream
        torch.cuda.current_stream().synchronize()
        _check("pp_server_submit", self._lib.pp_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (u, v, chi, usx, usy, points, normals, dS, p_out, per_point, forces)
        return rid.value

    def cancel(self, rid: int):
        _check("pp_server_cancel", self._lib.pp_server_cancel(self._h, int(rid)))

    def query(self, rid: int):
        st, err = ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_double * 3)()
        _check("pp_server_query", self._lib.pp_server_query(self._h, int(rid), ctypes.byref(st),
                                                            ctypes.byref(err), t))
        return st.value, err.value, (t[0], t[1], t[2])

    def wait(self, rid: int, timeout: float = 60.0) -> int:
        """pp_server_wait status (PP_OK, PP_ERR_TIMEOUT, ...); no exception."""
        st = self._lib.pp_server_wait(self._h, int(rid), float(timeout))
        if st == PP_OK:
            self._keep.pop(int(rid), None)
        return st

    def stats(self) -> dict:
        s = ServerStats()
        _check("pp_server_stats", self._lib.pp_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def destroy(self):
        if self._h and self._h.value:
            self._lib.pp_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


PP_NOALLOC_MAX_POINTS = 1 << 20


def pp_surface_forces_noalloc(u, v, points, normals, P_points, *, n: int, h: float, nu: float,
                              x0: float = 0.0, y0: float = 0.0, rho: float = 1.0, lift: float = None,
                              interp: str = "nearest", uinf=(1.0, 0.0), dS=None, per_point=None,
                              forces=None):
    """Tractions and drag/lift from a given surface pressure without any device
    allocation (for callers that cannot allocate; see include/pp.h).  Precision
    follows the dtype of u (float64: FP64, float32: mixed).  Returns the forces as
    a host array when ``forces`` is None."""
    import torch
    lib = load()
    prec = PP_FP64 if u.dtype == torch.float64 else PP_MIXED
    npts = int(points.shape[0])
    nn = int(n) * int(n)
    host = None
    if forces is None:
        host = np.zeros(6, np.float64)
        fptr = ctypes.c_void_p(host.ctypes.data)
    else:
        fptr = _dptr(forces, torch.float64, 6, "forces")
    st = lib.pp_surface_forces_noalloc(
        prec, _Grid(int(n), float(x0), float(y0)), float(h), _dptr(u, u.dtype, nn, "u"),
        _dptr(v, u.dtype, nn, "v"), npts, _dptr(points, torch.float64, 2 * npts, "points"),
        _dptr(normals, torch.float64, 2 * npts, "normals"), _dptr(dS, torch.float64, npts, "dS"),
        _dptr(P_points, torch.float64, npts, "P_points"), float(rho), float(nu),
        -1.0 if lift is None else float(lift), {"nearest": PP_NEAREST, "bilinear": PP_BILINEAR}[interp],
        float(uinf[0]), float(uinf[1]), _dptr(per_point, torch.float64, 5 * npts, "per_point"), fptr,
        _stream_ptr())
    _check("pp_surface_forces_noalloc", st)
    return host


# C-ABI-named convenience functions (same names as include/pp.h) ------------------
def pp_plan_create(n, h, order=20, theta=0.5, **kw) -> Plan:
    return Plan(n, h, order, theta, **kw)


def pp_rhs(plan: Plan, u, v, chi, usx, usy, lam, f_out=None):
    return plan.rhs(u, v, chi, usx, usy, lam, f_out)


def pp_pressure_solve(plan: Plan, p_out=None):
    return plan.pressure_solve(p_out)


def _atree_handle(level, ix, iy, theta: float, device: bool = False):
    """pp_atree_create (host build) or pp_atree_create_device (GPU build from device copies of
    the three arrays, on torch's current stream); returns (handle, leaf count)."""
    import numpy as np
    lib = load()
    ip = ctypes.POINTER(ctypes.c_int)
    lv, xs, ys = (np.ascontiguousarray(a, dtype=np.int32) for a in (level, ix, iy))
    if not (lv.shape == xs.shape == ys.shape and lv.ndim == 1):
        raise ValueError("level, ix and iy must be 1-D arrays of one length")
    h = ctypes.c_void_p()
    if device:
        import torch
        d = [torch.from_numpy(a).cuda() for a in (lv, xs, ys)]
        _check("pp_atree_create_device", lib.pp_atree_create_device(
            int(lv.size), *(ctypes.c_void_p(t.data_ptr()) for t in d), float(theta), _stream_ptr(), ctypes.byref(h)))
    else:
        _check("pp_atree_create", lib.pp_atree_create(int(lv.size), lv.ctypes.data_as(ip), xs.ctypes.data_as(ip),
                                                      ys.ctypes.data_as(ip), float(theta), ctypes.byref(h)))
    return h, int(lv.size)


def adaptive_tree(level, ix, iy, theta: float, device: bool = False) -> dict:
    """pp_atree_*: the adaptive quadtree over leaf blocks (level, ix, iy) tiling the unit
    domain and its dual-tree interaction lists, built on the host or (``device``) on the GPU.
    Returns numpy arrays: per box ``level, ix, iy, parent, first_child, leaf`` and the pair
    lists ``m2l`` (target box, source box) and ``p2p`` (target leaf, source leaf), each of
    shape (count, 2)."""
    import numpy as np
    lib = load()
    ip = ctypes.POINTER(ctypes.c_int)
    h, _ = _atree_handle(level, ix, iy, theta, device)
    try:
        sizes = (ctypes.c_int64 * 4)()
        _check("pp_atree_sizes", lib.pp_atree_sizes(h, sizes))
        nb, nm, npp = int(sizes[0]), int(sizes[1]), int(sizes[2])
        out = {k: np.empty(nb, np.int32) for k in ("level", "ix", "iy", "parent", "first_child", "leaf")}
        _check("pp_atree_boxes", lib.pp_atree_boxes(h, *(out[k].ctypes.data_as(ip) for k in
                                                         ("level", "ix", "iy", "parent", "first_child", "leaf"))))
        out["m2l"] = np.empty((nm, 2), np.int32)
        out["p2p"] = np.empty((npp, 2), np.int32)
        _check("pp_atree_lists", lib.pp_atree_lists(h, out["m2l"].ctypes.data_as(ip), out["p2p"].ctypes.data_as(ip)))
        out["max_level"] = int(sizes[3])
        return out
    finally:
        lib.pp_atree_destroy(h)


class AdaptiveTree:
    """pp_atree_*: an adaptive grid's tree and lists, kept for repeated solves.  The first
    solve uploads them and allocates the expansions; later solves only launch kernels (on
    torch's current stream; solves on one tree must be ordered, they share its arrays)."""

    def __init__(self, level, ix, iy, theta: float = 0.5, device: bool = False):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self._h, self.nleaf = _atree_handle(level, ix, iy, theta, device)

    def solve(self, q, order: int = 20, p_out=None):
        """pp_atree_solve: FP64 pressure at every cell.  q: CUDA float64 tensor of nleaf*64
        cell weights f h^2, leaf-major in the leaf order given, cell (cx, cy) at cy*8 + cx.
        Returns p_out (allocated if None)."""
        import torch
        nn = self.nleaf * 64
        if p_out is None:
            p_out = torch.empty(nn, dtype=torch.float64, device="cuda")
        _check("pp_atree_solve", self._lib.pp_atree_solve(self._h, int(order), _dptr(q, torch.float64, nn, "q"),
                                                          _dptr(p_out, torch.float64, nn, "p_out"), _stream_ptr()))
        return p_out

    def solve_mixed(self, q, order: int = 12, p_out=None):
        """pp_atree_solve_mixed: the same pressure in mixed precision.  q: CUDA float32 tensor
        of nleaf*64 cell weights (layout as in solve).  Returns p_out (float32, allocated if None)."""
        import torch
        nn = self.nleaf * 64
        if p_out is None:
            p_out = torch.empty(nn, dtype=torch.float32, device="cuda")
        _check("pp_atree_solve_mixed", self._lib.pp_atree_solve_mixed(
            self._h, int(order), _dptr(q, torch.float32, nn, "q"), _dptr(p_out, torch.float32, nn, "p_out"),
            _stream_ptr()))
        return p_out

    def surface_pressure(self, q, points, theta: float = 0.5, P_out=None):
        """pp_atree_surface_pressure: FP64 pressure at off-grid points (npts x 2 CUDA float64) by
        the tree-code over this tree, from the multipoles of the last solve (same q)."""
        import torch
        nn = self.nleaf * 64
        npts = int(points.shape[0])
        if P_out is None:
            P_out = torch.empty(npts, dtype=torch.float64, device="cuda")
        _check("pp_atree_surface_pressure", self._lib.pp_atree_surface_pressure(
            self._h, _dptr(q, torch.float64, nn, "q"), npts, _dptr(points, torch.float64, 2 * npts, "points"),
            float(theta), _dptr(P_out, torch.float64, npts, "P_out"), _stream_ptr()))
        return P_out

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pp_atree_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def adaptive_solve(level, ix, iy, q, theta: float = 0.5, order: int = 20, p_out=None):
    """One solve on a tree built for it (AdaptiveTree.solve, then the tree is released)."""
    import torch
    t = AdaptiveTree(level, ix, iy, theta)
    try:
        out = t.solve(q, order, p_out)
        torch.cuda.current_stream().synchronize()
        return out
    finally:
        t.destroy()


def pp_pressure_solve_fft(plan: Plan, p_out):
    return plan.pressure_solve_fft(p_out)


def pp_surface_traction(plan: Plan, u, v, points, normals, nu, dS=None, per_point=None, forces=None):
    return plan.surface_traction(u, v, points, normals, nu, dS, per_point, forces)


def pp_plan_destroy(plan: Plan):
    plan.destroy()
