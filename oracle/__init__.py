"""ctypes wrapper of the FP64 reference (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The library is plain C
compiled with ``gcc -O2 -ffp-contract=off`` so that it rounds the same way on
x86-64 and aarch64 hosts, and with OpenMP over the independent cell loops
(any thread count gives the same bits).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXC, MAXV = 4, 10


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no GPU needed)."""
    src_m = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < src_m:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Comp(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("pinf", C.c_double), ("cv", C.c_double),
                ("q", C.c_double), ("Tc", C.c_double), ("pc", C.c_double), ("omega", C.c_double),
                ("M", C.c_double), ("mu", C.c_double), ("kc", C.c_double), ("psat", C.c_double),
                ("rho_sl", C.c_double), ("rho_sv", C.c_double), ("cl", C.c_double), ("rt", C.c_double)]


class Params(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3), ("bc", (C.c_int * 2) * 3),
                ("ncomp", C.c_int), ("liquid", C.c_int), ("comp", Comp * MAXC),
                ("iles", C.c_int), ("thinc", C.c_int), ("beta", C.c_double), ("thinc_eps", C.c_double),
                ("thinc_gamma", C.c_double), ("lim_vel", C.c_int), ("lim_scalar", C.c_int),
                ("thr_ducros", C.c_double), ("thr_gas", C.c_double), ("eps_ducros", C.c_double),
                ("d3p_coef", C.c_double), ("sigma", C.c_double), ("grad_eps", C.c_double),
                ("in_yc", C.c_double), ("in_zc", C.c_double), ("in_radius", C.c_double),
                ("in_T", C.c_double), ("in_Y", C.c_double * MAXC), ("in_u", C.POINTER(C.c_double)),
                ("in_u0", C.c_double * 3), ("grav", C.c_double * 3), ("thr_vap", C.c_double),
                ("curv", C.c_int), ("st_model", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            P = C.POINTER(Params)
            L.or_closure_forward.argtypes = [P, C.c_double, C.c_double, dp, dp, dp, dp, dp]
            L.or_closure_inverse.argtypes = [P, C.c_double, C.c_double, dp, dp, dp]
            L.or_limiter.argtypes = [C.c_int, C.c_double]
            L.or_limiter.restype = C.c_double
            L.or_muscl.argtypes = [C.c_int] + [C.c_double] * 4 + [dp, dp]
            L.or_thinc.argtypes = [C.c_double] * 6 + [dp, dp]
            L.or_face_flux.argtypes = [P, C.c_int, dp, dp, dp, C.c_int, dp]
            L.or_prim_to_cons.argtypes = [P, dp, dp]
            L.or_cons_to_prim.argtypes = [P, dp, dp]
            L.or_stage.argtypes = [P, C.c_int, C.c_double, dp, dp, dp, ip, ip]
            L.or_dt.argtypes = [P, dp, C.c_double, dp]
            L.or_step.argtypes = [P, dp, C.c_int, C.c_double, dp]
            L.or_totals.argtypes = [P, dp, dp]
            L.or_csf_source.argtypes = [P, dp, dp]
            L.or_sensor.argtypes = [P, dp, dp]
            L.or_transport.argtypes = [P, dp, dp]
            L.or_curvature.argtypes = [P, dp, dp]
            L.or_sensor_args.argtypes = [P, dp, dp]
            L.or_hf_axis.argtypes = [P, dp, dp, dp]
            L.or_baro_vapour.argtypes = [P, C.c_double, dp]
            L.or_baro_vapour.restype = C.c_double
            L.or_face_flux_av.argtypes = [P, C.c_int, dp, dp, dp, dp, C.c_int, dp]
            L.or_pr_state.argtypes = [P, C.c_double, C.c_double, dp, dp]
            L.or_set_threads.argtypes = [C.c_int]
            L.or_smoothed_fraction.argtypes = [P, dp, dp]
            L.or_baro_sound_rho.argtypes = [P, C.c_double, C.c_double, dp, dp]
            L.or_capillary_force.argtypes = [P, dp, dp]
            L.or_face_flux_kappa.argtypes = [P, C.c_int, dp, dp, dp, C.c_int, C.c_double, C.c_double, dp, dp, dp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what}: oracle status {st}")


def make_params(w, inflow_u: np.ndarray | None = None) -> Params:
    """or_params from a workload description (paper_2304_00140_gb300.workloads)."""
    P = Params()
    P.ndim = w.ndim
    for d in range(3):
        P.n[d] = w.n[d]
        P.dx[d] = w.dx[d]
        P.bc[d][0], P.bc[d][1] = w.bc[d]
    P.ncomp = len(w.comps)
    P.liquid = w.liquid
    for k, c in enumerate(w.comps):
        P.comp[k] = Comp(c["kind"], c["gamma"], c["pinf"], c["cv"], c["q"], c["Tc"], c["pc"], c["omega"], c["M"],
                         c.get("mu", 0.0), c.get("kc", 0.0), c.get("psat", 0.0), c.get("rho_sl", 0.0),
                         c.get("rho_sv", 0.0), c.get("cl", 0.0), c.get("rt", 0.0))
    s = w.scheme
    P.iles, P.thinc = int(s["iles"]), int(s["thinc"])
    P.beta, P.thinc_eps, P.thinc_gamma = s["beta"], s["thinc_eps"], s["thinc_gamma"]
    P.lim_vel, P.lim_scalar = s["lim_vel"], s["lim_scalar"]
    P.thr_ducros, P.thr_gas, P.eps_ducros, P.d3p_coef = s["thr_ducros"], s["thr_gas"], s["eps_ducros"], s["d3p_coef"]
    P.sigma, P.grad_eps = s["sigma"], s["grad_eps"]
    for d, g in enumerate(s.get("gravity", (0.0, 0.0, 0.0))):
        P.grav[d] = g
    P.thr_vap = s.get("thr_vap", 0.4)
    P.curv = int(s.get("curvature", 0))
    P.st_model = int(s.get("st_model", 0))
    if w.inflow:
        f = w.inflow
        P.in_yc, P.in_zc, P.in_radius, P.in_T = f["yc"] - w.lo[1], f["zc"] - w.lo[2], f["radius"], f["T"]
        for k, y in enumerate(f["Y"]):
            P.in_Y[k] = y
        for d, u in enumerate(f.get("u0", (0.0, 0.0, 0.0))):
            P.in_u0[d] = u
    return P


class Oracle:
    """The FP64 reference on one workload.  Arrays are [nv, nz, ny, nx] float64."""

    def __init__(self, w, inflow_u: np.ndarray | None = None):
        self.w = w
        self.P = make_params(w)
        self._in_u = None
        if inflow_u is not None:
            self._in_u = np.ascontiguousarray(inflow_u, dtype=np.float64)
            self.P.in_u = _ptr(self._in_u)
        self.L = lib()
        self.shape = (w.nvar, w.n[2], w.n[1], w.n[0])

    def _new(self):
        return np.zeros(self.shape, dtype=np.float64)

    def prim_to_cons(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        q = self._new()
        _check(self.L.or_prim_to_cons(C.byref(self.P), _ptr(W), _ptr(q)), "prim_to_cons")
        return q

    def cons_to_prim(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        W = self._new()
        _check(self.L.or_cons_to_prim(C.byref(self.P), _ptr(q), _ptr(W)), "cons_to_prim")
        return W

    def stage(self, k, dt, q0, qprev, window=None, out=None):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        qprev = np.ascontiguousarray(qprev, dtype=np.float64)
        out = q0.copy() if out is None else out
        lo = hi = None
        if window is not None:
            lo = (C.c_int * 3)(*window[0])
            hi = (C.c_int * 3)(*window[1])
        _check(self.L.or_stage(C.byref(self.P), k, dt, _ptr(q0), _ptr(qprev), _ptr(out), lo, hi), "stage")
        return out

    def dt(self, q, cfl):
        q = np.ascontiguousarray(q, dtype=np.float64)
        r = C.c_double()
        _check(self.L.or_dt(C.byref(self.P), _ptr(q), cfl, C.byref(r)), "dt")
        return r.value

    def step(self, q, nsteps, cfl, t=0.0):
        q = np.array(q, dtype=np.float64, copy=True, order="C")
        tt = C.c_double(t)
        _check(self.L.or_step(C.byref(self.P), _ptr(q), nsteps, cfl, C.byref(tt)), "step")
        return q, tt.value

    def totals(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(self.w.nvar)
        self.L.or_totals(C.byref(self.P), _ptr(q), _ptr(out))
        return out

    def csf_source(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        S = np.zeros((self.w.ndim + 1,) + self.shape[1:])
        _check(self.L.or_csf_source(C.byref(self.P), _ptr(q), _ptr(S)), "csf_source")
        return S

    def transport(self, q):
        """mixture viscosity and conductivity per interior cell, [2, nz, ny, nx]"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((2,) + self.shape[1:])
        _check(self.L.or_transport(C.byref(self.P), _ptr(q), _ptr(out)), "transport")
        return out

    def curvature(self, q):
        """curvature the CSF source uses, per interior cell [nz, ny, nx]"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        k = np.zeros(self.shape[1:])
        _check(self.L.or_curvature(C.byref(self.P), _ptr(q), _ptr(k)), "curvature")
        return k

    def smoothed_fraction(self, q):
        """Gaussian-smoothed liquid fraction per interior cell [nz, ny, nx] (Eq. 3-9)"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        a = np.zeros(self.shape[1:])
        _check(self.L.or_smoothed_fraction(C.byref(self.P), _ptr(q), _ptr(a)), "smoothed_fraction")
        return a

    def baro_sound_rho(self, p, rho, Yt):
        """sound speed of a barotropic face state (p, rho, xi)"""
        Y = np.ascontiguousarray(Yt, dtype=np.float64)
        c = C.c_double()
        _check(self.L.or_baro_sound_rho(C.byref(self.P), p, rho, _ptr(Y), C.byref(c)), "baro_sound_rho")
        return c.value

    def sensor_args(self, q):
        """App. D switch arguments per interior cell (Eq. D.4):
        [theta^D, theta^Gas, theta^alpha, |div u|, |curl u|] x [nz, ny, nx]"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((5,) + self.shape[1:])
        _check(self.L.or_sensor_args(C.byref(self.P), _ptr(q), _ptr(out)), "sensor_args")
        return out

    def hf_axis(self, q):
        """height-function column axis per interior cell and the relative gap
        to the competing axis (Sec. 3.5 option)"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        axis = np.zeros(self.shape[1:])
        gap = np.zeros(self.shape[1:])
        _check(self.L.or_hf_axis(C.byref(self.P), _ptr(q), _ptr(axis), _ptr(gap)), "hf_axis")
        return axis.astype(int), gap

    def capillary_force(self, q):
        """momentum source of the capillary face jumps per interior cell,
        [ndim, nz, ny, nx] (st_model = 1)"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        S = np.zeros((self.w.ndim,) + self.shape[1:])
        _check(self.L.or_capillary_force(C.byref(self.P), _ptr(q), _ptr(S)), "capillary_force")
        return S

    def face_flux_kappa(self, d, W4, kapL, kapR, alpha2, rho4=None, c4=None, f=1):
        """one face with the capillary jump (st_model = 1) between cells of
        curvatures kapL, kapR and liquid fractions alpha2: (F, G)"""
        W = np.zeros((4, MAXV))
        W4 = np.asarray(W4, dtype=np.float64)
        W[:, :W4.shape[1]] = W4
        r4 = np.ascontiguousarray(rho4 if rho4 is not None else np.ones(4), dtype=np.float64)
        c4 = np.ascontiguousarray(c4 if c4 is not None else np.ones(4), dtype=np.float64)
        F, G = np.zeros(MAXV), np.zeros(2)
        a2 = np.ascontiguousarray(alpha2, dtype=np.float64)
        _check(self.L.or_face_flux_kappa(C.byref(self.P), d, _ptr(W), _ptr(r4), _ptr(c4), int(f), kapL, kapR,
                                         _ptr(a2), _ptr(F), _ptr(G)), "face_flux_kappa")
        return F[:self.w.nvar].copy(), G

    def sensor(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        f = np.zeros(self.shape[1:])
        _check(self.L.or_sensor(C.byref(self.P), _ptr(q), _ptr(f)), "sensor")
        return f

    # ---- pointwise ----
    def forward(self, p, T, Yt):
        Y = np.ascontiguousarray(Yt, dtype=np.float64)
        r, e, c = C.c_double(), C.c_double(), C.c_double()
        al = np.zeros(MAXC)
        _check(self.L.or_closure_forward(C.byref(self.P), p, T, _ptr(Y), C.byref(r), C.byref(e), C.byref(c),
                                         _ptr(al)), "forward")
        return r.value, e.value, c.value, al[:len(self.w.comps)].copy()

    def inverse(self, rho, e, Yt):
        Y = np.ascontiguousarray(Yt, dtype=np.float64)
        p, T = C.c_double(), C.c_double()
        _check(self.L.or_closure_inverse(C.byref(self.P), rho, e, _ptr(Y), C.byref(p), C.byref(T)), "inverse")
        return p.value, T.value

    def pr_state(self, T, v, Yt):
        Y = np.ascontiguousarray(Yt, dtype=np.float64)
        out = np.zeros(8)
        _check(self.L.or_pr_state(C.byref(self.P), T, v, _ptr(Y), _ptr(out)), "pr_state")
        return dict(p=out[0], e=out[1], c=out[2], cv=out[3], a=out[4], b=out[5], M=out[6], da=out[7])

    def vapour(self, p, alpha):
        """Eq. 2-7 vapour volume fraction at p given the phase fractions"""
        a = np.zeros(MAXC)
        a[:len(alpha)] = alpha
        return self.L.or_baro_vapour(C.byref(self.P), p, _ptr(a))

    def face_flux(self, d, W4, rho4=None, c4=None, f=1, av4=None):
        if av4 is not None:
            W = np.zeros((4, MAXV))
            W4 = np.asarray(W4, dtype=np.float64)
            W[:, :W4.shape[1]] = W4
            r4 = np.ascontiguousarray(rho4, dtype=np.float64)
            c4 = np.ascontiguousarray(c4 if c4 is not None else np.ones(4), dtype=np.float64)
            a4 = np.ascontiguousarray(av4, dtype=np.float64)
            F = np.zeros(MAXV)
            _check(self.L.or_face_flux_av(C.byref(self.P), d, _ptr(W), _ptr(r4), _ptr(c4), _ptr(a4), int(f),
                                          _ptr(F)), "face_flux_av")
            return F[:self.w.nvar].copy()
        W = np.zeros((4, MAXV))
        W4 = np.asarray(W4, dtype=np.float64)
        W[:, :W4.shape[1]] = W4
        r4 = np.ascontiguousarray(rho4 if rho4 is not None else np.ones(4), dtype=np.float64)
        c4 = np.ascontiguousarray(c4 if c4 is not None else np.ones(4), dtype=np.float64)
        F = np.zeros(MAXV)
        _check(self.L.or_face_flux(C.byref(self.P), d, _ptr(W), _ptr(r4), _ptr(c4), int(f), _ptr(F)), "face_flux")
        return F[:self.w.nvar].copy()


_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "libopcount.so")
_opc = None
OPCOUNT_CLASSES = ("add", "mul", "div", "sqrt", "minmax", "cmp", "abs", "transcendental")


def build_opcount(force: bool = False) -> str:
    """Compile the op-counting build of the oracle (g++, serial)."""
    src_m = max(os.path.getmtime(_OPC_SRC), os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if force or not os.path.exists(_OPC_LIB) or os.path.getmtime(_OPC_LIB) < src_m:
        tmp = _OPC_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-fpermissive", "-w",
                               "-ffp-contract=off", "-o", tmp, _OPC_SRC, "-lm"], cwd=_HERE)
        os.replace(tmp, _OPC_LIB)
    return _OPC_LIB


def opcount_stage(o: "Oracle", k, dt, q0, qprev):
    """One oracle stage with its arithmetic counted: (q^k, {class: count}
    of the stage, {class: count} of its boundary and primitive update)."""
    global _opc
    with _lock:
        if _opc is None:
            build_opcount()
            L = C.CDLL(_OPC_LIB)
            dp = C.POINTER(C.c_double)
            L.oc_stage.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp, dp, C.POINTER(C.c_ulonglong)]
            L.oc_box_fill.argtypes = [C.c_void_p, dp, C.POINTER(C.c_ulonglong)]
            _opc = L
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    qprev = np.ascontiguousarray(qprev, dtype=np.float64)
    out = q0.copy()
    cnt = (C.c_ulonglong * len(OPCOUNT_CLASSES))()
    _check(_opc.oc_stage(C.cast(C.byref(o.P), C.c_void_p), k, dt, _ptr(q0), _ptr(qprev), _ptr(out), cnt),
           "opcount stage")
    out_counts = dict(zip(OPCOUNT_CLASSES, [int(c) for c in cnt]))
    _check(_opc.oc_box_fill(C.cast(C.byref(o.P), C.c_void_p), _ptr(qprev), cnt), "opcount box")
    return out, out_counts, dict(zip(OPCOUNT_CLASSES, [int(c) for c in cnt]))


def threads(n: int = 0) -> int:
    """threads of the oracle's cell loops (OpenMP); n < 1 only reports the
    count.  Cells are independent, so every count gives the same bits."""
    return lib().or_set_threads(int(n))


def limiter(lim_id, r):
    return lib().or_limiter(lim_id, r)


def muscl(lim_id, x1, x2, x3, x4):
    L, R = C.c_double(), C.c_double()
    lib().or_muscl(lim_id, x1, x2, x3, x4, C.byref(L), C.byref(R))
    return L.value, R.value


def thinc(beta, gam, x1, x2, x3, x4):
    L, R = C.c_double(), C.c_double()
    lib().or_thinc(beta, gam, x1, x2, x3, x4, C.byref(L), C.byref(R))
    return L.value, R.value
