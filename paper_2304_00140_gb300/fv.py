"""Python binding of the C ABI in include/thinc_fv.h (argument marshalling
only -- every step of the stage runs in the CUDA kernels of libthinc_fv.so).

PyTorch supplies the device workspace and the stream.  There is no CPU
fallback: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional

import numpy as np

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthinc_fv.so")
MAX_COMP = 3

FV_OK, FV_ERR_ARG, FV_ERR_ALLOC, FV_ERR_CUDA, FV_ERR_EOS_NONCONV, FV_ERR_NONPHYSICAL, FV_ERR_STATE = range(7)
FV_FP64, FV_MIXED = 0, 1
FV_CONSERVED, FV_PRIMITIVE = 0, 1
FV_DIAG_TOTALS, FV_DIAG_DT, FV_DIAG_TIME, FV_DIAG_ERROR, FV_DIAG_TILE, FV_DIAG_FLAGS = range(6)

# every exported function of the ABI (checked against include/thinc_fv.h by the tests)
EXPORTS = ["fv_workspace_size", "fv_init", "fv_init_ws", "fv_destroy", "fv_set_stream", "fv_set_state",
           "fv_get_state", "fv_set_state_device", "fv_get_state_device", "fv_rk_stage", "fv_step",
           "fv_step_async", "fv_get_diag", "fv_launch_count", "fv_last_error", "fv_status_string",
           "fv_profile", "fv_profile_read", "fv_rk_stage_noalloc", "fv_set_state_all", "fv_get_state_all",
           "fv_wait_selftest", "fv_probe_fp64", "fv_split_workspace_size", "fv_init_split", "fv_upload_async",
           "fv_commit_upload", "fv_download_async", "fv_io_wait"]
FV_KERNEL_PRIM, FV_KERNEL_DT, FV_KERNEL_STAGE = range(3)


class fv_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3), ("in_yc", C.c_double), ("in_zc", C.c_double),
                ("in_radius", C.c_double), ("in_T", C.c_double), ("in_u0", C.c_double * 3),
                ("in_Y", C.c_double * MAX_COMP), ("in_u", C.POINTER(C.c_double))]


class fv_component(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("pinf", C.c_double), ("cv", C.c_double),
                ("q", C.c_double), ("Tc", C.c_double), ("pc", C.c_double), ("omega", C.c_double),
                ("M", C.c_double), ("mu", C.c_double), ("kc", C.c_double), ("psat", C.c_double),
                ("rho_sl", C.c_double), ("rho_sv", C.c_double), ("cl", C.c_double), ("rt", C.c_double)]


class fv_components(C.Structure):
    _fields_ = [("ncomp", C.c_int), ("liquid", C.c_int), ("comp", fv_component * MAX_COMP)]


class fv_eos(C.Structure):
    _fields_ = [("iles", C.c_int), ("thinc", C.c_int), ("beta", C.c_double), ("thinc_eps", C.c_double),
                ("thinc_gamma", C.c_double), ("lim_vel", C.c_int), ("lim_scalar", C.c_int),
                ("thr_ducros", C.c_double), ("thr_gas", C.c_double), ("eps_ducros", C.c_double),
                ("d3p_coef", C.c_double), ("sigma", C.c_double), ("grad_eps", C.c_double),
                ("precision", C.c_int), ("p_ref", C.c_double), ("T_ref", C.c_double),
                ("gravity", C.c_double * 3), ("thr_vap", C.c_double), ("curvature", C.c_int),
                ("st_model", C.c_int)]


_lock = threading.Lock()
_lib = None


class FVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def load(build_if_missing: bool = True):
    """Load libthinc_fv.so (building it in-tree first when asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _b
            _b.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run paper_2304_00140_gb300.build)")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        G, CM, E = C.POINTER(fv_grid), C.POINTER(fv_components), C.POINTER(fv_eos)
        L.fv_workspace_size.argtypes = [C.c_int, G, CM, E, C.POINTER(C.c_size_t)]
        L.fv_init.argtypes = [C.c_int, G, CM, E, C.POINTER(vp)]
        L.fv_init_ws.argtypes = [C.c_int, G, CM, E, vp, C.c_size_t, C.POINTER(vp)]
        L.fv_destroy.argtypes = [vp]
        L.fv_destroy.restype = None
        L.fv_set_stream.argtypes = [vp, vp]
        for f in ("fv_set_state", "fv_get_state", "fv_set_state_device", "fv_get_state_device"):
            getattr(L, f).argtypes = [vp, C.c_int, C.c_int, vp]
        for f in ("fv_set_state_all", "fv_get_state_all"):
            getattr(L, f).argtypes = [vp, C.c_int, vp]
        L.fv_wait_selftest.argtypes = [C.c_int, C.POINTER(C.c_int)]
        ip = C.POINTER(C.c_int)
        L.fv_split_workspace_size.argtypes = [G, C.c_int, ip, CM, E, C.POINTER(C.c_size_t)]
        L.fv_init_split.argtypes = [G, C.c_int, ip, CM, E, vp, C.c_size_t, C.POINTER(vp)]
        L.fv_probe_fp64.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        for f in ("fv_upload_async", "fv_download_async"):
            getattr(L, f).argtypes = [vp, vp]
        for f in ("fv_commit_upload", "fv_io_wait"):
            getattr(L, f).argtypes = [vp]
        L.fv_rk_stage.argtypes = [vp, C.c_int, C.c_double]
        L.fv_step.argtypes = [vp, C.c_int, C.c_double, dp]
        L.fv_step_async.argtypes = [vp, C.c_int, C.c_double]
        L.fv_get_diag.argtypes = [vp, C.c_int, C.c_int, vp]
        L.fv_launch_count.argtypes = [vp]
        L.fv_launch_count.restype = C.c_longlong
        L.fv_last_error.argtypes = [vp]
        L.fv_last_error.restype = C.c_char_p
        L.fv_profile.argtypes = [vp, C.c_int]
        L.fv_profile_read.argtypes = [vp, dp]
        L.fv_rk_stage_noalloc.argtypes = [G, CM, E, C.c_int, C.c_double, vp, vp, vp, vp]
        L.fv_status_string.argtypes = [C.c_int]
        L.fv_status_string.restype = C.c_char_p
        _lib = L
        return L


def status_string(s: int) -> str:
    try:
        return load(False).fv_status_string(s).decode()
    except Exception:
        return f"status {s}"


# ------------------------------------------------------------ marshalling
def make_grid(w: "wl.Workload") -> fv_grid:
    g = fv_grid()
    g.ndim = w.ndim
    for d in range(3):
        g.n[d] = w.n[d]
        g.lo[d] = w.lo[d]
        g.hi[d] = w.hi[d]
        g.bc[d][0], g.bc[d][1] = w.bc[d]
    if w.inflow:
        f = w.inflow
        g.in_yc, g.in_zc, g.in_radius, g.in_T = f["yc"], f["zc"], f["radius"], f["T"]
        for d, u in enumerate(f.get("u0", (0.0, 0.0, 0.0))):
            g.in_u0[d] = u
        for k, y in enumerate(f["Y"]):
            g.in_Y[k] = y
    return g


def make_components(w: "wl.Workload") -> fv_components:
    c = fv_components()
    c.ncomp = len(w.comps)
    c.liquid = w.liquid
    for k, m in enumerate(w.comps):
        c.comp[k] = fv_component(m["kind"], m["gamma"], m["pinf"], m["cv"], m["q"], m["Tc"], m["pc"], m["omega"], m["M"],
                                 m.get("mu", 0.0), m.get("kc", 0.0), m.get("psat", 0.0), m.get("rho_sl", 0.0),
                                 m.get("rho_sv", 0.0), m.get("cl", 0.0), m.get("rt", 0.0))
    return c


def make_eos(s: dict) -> fv_eos:
    e = fv_eos()
    e.iles, e.thinc = int(s["iles"]), int(s["thinc"])
    e.beta, e.thinc_eps, e.thinc_gamma = s["beta"], s["thinc_eps"], s["thinc_gamma"]
    e.lim_vel, e.lim_scalar = int(s["lim_vel"]), int(s["lim_scalar"])
    e.thr_ducros, e.thr_gas, e.eps_ducros, e.d3p_coef = s["thr_ducros"], s["thr_gas"], s["eps_ducros"], s["d3p_coef"]
    e.sigma, e.grad_eps = s["sigma"], s["grad_eps"]
    e.precision = int(s["precision"])
    e.p_ref, e.T_ref = s["p_ref"], s["T_ref"]
    for d, g in enumerate(s.get("gravity", (0.0, 0.0, 0.0))):
        e.gravity[d] = g
    e.thr_vap = s.get("thr_vap", 0.4)
    e.curvature = int(s.get("curvature", 0))
    e.st_model = int(s.get("st_model", 0))
    return e


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


class Solver:
    """One context over one workload or a list of workloads (a batch).

    Device memory is one torch uint8 tensor handed to fv_init_ws; the context
    runs on torch's current CUDA stream.
    """

    def __init__(self, cases, precision: Optional[int] = None, inflow_u: Optional[List[np.ndarray]] = None,
                 split: Optional[tuple] = None):
        """split = (nblocks, rows or None): one grid (a single workload) as
        slabs along its last dimension (fv_init_split); the cases are then
        the slabs and set_state_grid / get_state_grid move the whole grid."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the THINC-TDU solver needs a CUDA device")
        self.L = load()
        self.cases = list(cases) if isinstance(cases, (list, tuple)) else [cases]
        w0 = self.cases[0]
        scheme = dict(w0.scheme)
        if precision is not None:
            scheme["precision"] = precision
        self.precision = scheme["precision"]
        self._comps = make_components(w0)
        self._eos = make_eos(scheme)
        self._in_u = []
        nbytes = C.c_size_t()
        ctx = C.c_void_p()
        if split is not None:
            import dataclasses

            from . import slabs
            assert len(self.cases) == 1
            nb, rows = split
            ax = w0.ndim - 1
            self.slabs = slabs.plan(w0.n[ax], nb, rows, periodic=w0.bc[ax][0] == wl.BC_PERIODIC)
            g = make_grid(w0)
            if inflow_u is not None and inflow_u[0] is not None:
                a = np.ascontiguousarray(inflow_u[0], dtype=np.float64)
                self._in_u.append(a)
                g.in_u = a.ctypes.data_as(C.POINTER(C.c_double))
            rr = (C.c_int * nb)(*[s["rows"] for s in self.slabs])
            self._check(self.L.fv_split_workspace_size(C.byref(g), nb, rr, C.byref(self._comps), C.byref(self._eos),
                                                       C.byref(nbytes)), None)
            self.ws = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device="cuda")
            st = self.L.fv_init_split(C.byref(g), nb, rr, C.byref(self._comps), C.byref(self._eos),
                                      C.c_void_p(self.ws.data_ptr()), nbytes.value, C.byref(ctx))
            self.grid = w0
            self.cases = [dataclasses.replace(w0, n=[s["rows"] if d == ax else w0.n[d] for d in range(3)])
                          for s in self.slabs]
        else:
            n = len(self.cases)
            self._grids = (fv_grid * n)()
            for i, w in enumerate(self.cases):
                self._grids[i] = make_grid(w)
                if inflow_u is not None and inflow_u[i] is not None:
                    a = np.ascontiguousarray(inflow_u[i], dtype=np.float64)
                    self._in_u.append(a)
                    self._grids[i].in_u = a.ctypes.data_as(C.POINTER(C.c_double))
            self._check(self.L.fv_workspace_size(n, self._grids, C.byref(self._comps), C.byref(self._eos),
                                                 C.byref(nbytes)), None)
            self.ws = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device="cuda")
            st = self.L.fv_init_ws(n, self._grids, C.byref(self._comps), C.byref(self._eos),
                                   C.c_void_p(self.ws.data_ptr()), nbytes.value, C.byref(ctx))
        self.ctx = ctx
        self._check(st)
        self.set_stream(torch.cuda.current_stream().cuda_stream)

    # -- plumbing
    def _check(self, st, ctx="self"):
        if st != FV_OK:
            msg = ""
            c = self.ctx if ctx == "self" else ctx
            if c:
                msg = self.L.fv_last_error(c).decode()
            raise FVError(st, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.L.fv_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int):
        self._check(self.L.fv_set_stream(self.ctx, C.c_void_p(stream_handle)))

    # -- state
    def shape(self, i=0):
        w = self.cases[i]
        return (w.nvar, w.n[2], w.n[1], w.n[0])

    def set_state(self, arr: np.ndarray, kind=FV_CONSERVED, case: int = 0):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.size == int(np.prod(self.shape(case)))
        self._check(self.L.fv_set_state(self.ctx, case, kind, _dptr(a)))

    def get_state(self, kind=FV_CONSERVED, case: int = 0) -> np.ndarray:
        a = np.zeros(self.shape(case), dtype=np.float64)
        self._check(self.L.fv_get_state(self.ctx, case, kind, _dptr(a)))
        return a

    def set_state_device(self, t, kind=FV_CONSERVED, case: int = 0):
        self._check(self.L.fv_set_state_device(self.ctx, case, kind, C.c_void_p(t.data_ptr())))

    def get_state_device(self, t, kind=FV_CONSERVED, case: int = 0):
        self._check(self.L.fv_get_state_device(self.ctx, case, kind, C.c_void_p(t.data_ptr())))

    def _slab_axis(self):
        return 3 - (self.grid.ndim - 1)

    def set_state_grid(self, arr: np.ndarray, kind=FV_CONSERVED):
        """a split context: the whole grid's [nv, nz, ny, nx] state, slab by slab"""
        ax = self._slab_axis()
        for b, s in enumerate(self.slabs):
            self.set_state(np.take(arr, np.arange(s["row0"], s["row0"] + s["rows"]), axis=ax), kind, case=b)

    def get_state_grid(self, kind=FV_CONSERVED) -> np.ndarray:
        return np.concatenate([self.get_state(kind, case=b) for b in range(len(self.slabs))],
                              axis=self._slab_axis())

    def set_state_all(self, arr: np.ndarray, kind=FV_CONSERVED):
        """every case at once: each case's state flattened, concatenated in case order"""
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.size == sum(int(np.prod(self.shape(c))) for c in range(len(self.cases)))
        self._check(self.L.fv_set_state_all(self.ctx, kind, _dptr(a)))

    def get_state_all(self, kind=FV_CONSERVED) -> np.ndarray:
        a = np.zeros(sum(int(np.prod(self.shape(c))) for c in range(len(self.cases))), dtype=np.float64)
        self._check(self.L.fv_get_state_all(self.ctx, kind, _dptr(a)))
        return a

    # -- time stepping
    def rk_stage(self, k: int, dt: float):
        self._check(self.L.fv_rk_stage(self.ctx, k, dt))

    def step_dt(self, dt: float):
        for k in (1, 2, 3, 4):
            self.rk_stage(k, dt)

    def step(self, nsteps: int, cfl: float) -> float:
        t = C.c_double()
        self._check(self.L.fv_step(self.ctx, nsteps, cfl, C.byref(t)))
        return t.value

    def step_async(self, nsteps: int, cfl: float):
        self._check(self.L.fv_step_async(self.ctx, nsteps, cfl))

    # -- diagnostics
    def totals(self, case=0) -> np.ndarray:
        out = np.zeros(self.cases[case].nvar)
        self._check(self.L.fv_get_diag(self.ctx, case, FV_DIAG_TOTALS, _dptr(out)))
        return out

    def diag_scalar(self, what, case=0) -> float:
        out = np.zeros(1)
        self._check(self.L.fv_get_diag(self.ctx, case, what, _dptr(out)))
        return float(out[0])

    def tile(self) -> dict:
        out = np.zeros(12)
        self._check(self.L.fv_get_diag(self.ctx, 0, FV_DIAG_TILE, _dptr(out)))
        return dict(tile=[int(v) for v in out[:3]], threads=int(out[3]), tune_ms=out[4:8].tolist(),
                    fused=bool(out[8] == 1), zmarch=bool(out[8] == 2), fused_ms=float(out[9]),
                    prim_ms=float(out[10]), fused_variant=int(out[11]))

    def sensor_flags(self, case: int = 0) -> np.ndarray:
        """App. D sensor flag (0/1) of every interior cell, [nz, ny, nx] uint8"""
        w = self.cases[case]
        out = np.zeros((w.n[2], w.n[1], w.n[0]), dtype=np.uint8)
        self._check(self.L.fv_get_diag(self.ctx, case, FV_DIAG_FLAGS, C.c_void_p(out.ctypes.data)))
        return out

    def error_word(self) -> int:
        out = C.c_int()
        self._check(self.L.fv_get_diag(self.ctx, 0, FV_DIAG_ERROR, C.byref(out)))
        return out.value

    def launch_count(self) -> int:
        return int(self.L.fv_launch_count(self.ctx))

    def profile(self, enable: bool):
        self._check(self.L.fv_profile(self.ctx, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = np.zeros(6)
        self._check(self.L.fv_profile_read(self.ctx, out.ctypes.data_as(C.POINTER(C.c_double))))
        names = ("prim", "dt", "stage")
        return {n: dict(ms=float(out[2 * i]), launches=int(out[2 * i + 1])) for i, n in enumerate(names)}
