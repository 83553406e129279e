"""fv_rk_stage_noalloc: the stage entry point for callers that cannot
allocate device memory (a host application that owns the device through its
own pool, a fixed memory budget, or a path where an allocation is not
allowed).  It must give the same result as fv_rk_stage, call after call, and
refuse grids whose scratch does not fit its static array.

This file is collected last on purpose: it runs alone in a fresh process as
well as after every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import rel_field_diff

pytestmark = pytest.mark.gpu


def _abi(w, precision):
    g = fv.make_grid(w)
    cm = fv.make_components(w)
    e = fv.make_eos(dict(w.scheme, precision=precision))
    return g, cm, e


def _noalloc_step(L, args, dt, q0, qa, qb, stream):
    g, cm, e = args
    regs = [(q0, q0, qa), (q0, qa, qb), (q0, qb, qa), (q0, qa, q0)]
    for k, (base, prev, out) in enumerate(regs, start=1):
        st = L.fv_rk_stage_noalloc(C.byref(g), C.byref(cm), C.byref(e), k, dt, C.c_void_p(base.data_ptr()),
                                   C.c_void_p(prev.data_ptr()), C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert st == fv.FV_OK, fv.status_string(st)


# max relative difference per field: the FP64 form's parity tolerance; in the
# FP32-mixed form the context keeps float-float registers while the no-alloc
# call works on the caller's FP64 arrays, so the two agree to the mixed
# form's tolerance
TOL = {fv.FV_FP64: 1e-12, fv.FV_MIXED: 1e-6}


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
@pytest.mark.parametrize("lims,viscous", [((wl.LIM_KOREN, wl.LIM_MINMOD), False), ((wl.LIM_VANLEER, wl.LIM_MC), False),
                                          ((wl.LIM_KOREN, wl.LIM_MINMOD), True)])
def test_noalloc_matches_fv_rk_stage_twice(precision, lims, viscous):
    import torch
    w = wl.random_state(n=(37, 23), bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2, [0, 0]],
                        lim_vel=lims[0], lim_scalar=lims[1])
    if viscous:   # stress, heat flux and gravity terms (Eq. 2-2)
        w = wl.with_transport(w, mu=[2e-3, 5e-3], kc=[0.4, 0.6], gravity=(0.3, -9.8, 0.0))
    s = fv.Solver(w, precision=precision)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    q = s.get_state()
    dt = 0.2 * 0.4 / (np.abs(q[1] / q[0]).max() / w.dx[0] + 5000.0 / w.dx[0])
    refs = []
    for _ in range(2):
        s.step_dt(dt)
        refs.append(s.get_state())
    L = fv.load()
    args = _abi(w, precision)
    q0 = torch.from_numpy(q.copy()).cuda()
    qa, qb = torch.empty_like(q0), torch.empty_like(q0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        _noalloc_step(L, args, dt, q0, qa, qb, stream)
        got = q0.cpu().numpy()
        d = rel_field_diff(got, refs[call])
        assert np.all(d <= TOL[precision]), (call, d)


def test_noalloc_barotropic_fp64_matches_fv_rk_stage():
    """the barotropic closure through the no-alloc entry point (FP64 form)"""
    import torch
    w = wl.bubble_collapse("vapour", n=(64, 60))
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    q = s.get_state()
    dt = 2e-10
    s.step_dt(dt)
    ref = s.get_state()
    L = fv.load()
    args = _abi(w, fv.FV_FP64)
    q0 = torch.from_numpy(q.copy()).cuda()
    qa, qb = torch.empty_like(q0), torch.empty_like(q0)
    _noalloc_step(L, args, dt, q0, qa, qb, torch.cuda.current_stream().cuda_stream)
    d = rel_field_diff(q0.cpu().numpy(), ref)
    assert np.all(d <= 1e-12), d
    g, cm, e = _abi(w, fv.FV_MIXED)            # the mixed no-alloc variants are stiffened-gas only
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    st = L.fv_rk_stage_noalloc(C.byref(g), C.byref(cm), C.byref(e), 1, dt, p, p, p,
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fv.FV_ERR_ARG


def _inflow_jet(n):
    """the jet's inflow disc with a uniform inflow velocity (the no-alloc
    call takes no per-cell inflow array)"""
    return wl.jet3d(n=n, steps=1)


SCHEMES = {
    "3d_plain_periodic": lambda: wl.random_state(n=(20, 14, 11), ndim=3),
    "3d_iles_csf_3comp": lambda: wl.random_state(n=(18, 13, 12), ndim=3, ncomp=3, iles=1, sigma=5.0),
    "2d_csf_smoothed_normals": lambda: wl.droplet(n=(40, 36), A=0.15, sigma=30.0),
    "2d_csf_height_function": lambda: wl.droplet(n=(40, 36), A=0.15, sigma=30.0, curvature=1),
    "2d_iles_csf_3comp": lambda: wl.random_state(n=(33, 29), ncomp=3, iles=1, sigma=5.0),
    "3d_inflow_disc": lambda: _inflow_jet((24, 16, 16)),
}


@pytest.mark.parametrize("name", sorted(SCHEMES))
def test_noalloc_scheme_options_match_fv_rk_stage(name):
    """3D grids, CSF with both curvature options (Sec. 3.5), the App. D
    switch and the inflow disc through the no-alloc entry point, FP64, two
    steps in a row against the context path"""
    import torch
    w = SCHEMES[name]()
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    s.step(5 if w.inflow else 1, w.cfl)     # (the jet enters the domain first)
    q = s.get_state()
    dt = 0.3 * s.diag_scalar(fv.FV_DIAG_DT)
    refs = []
    for _ in range(2):
        s.step_dt(dt)
        refs.append(s.get_state())
    L = fv.load()
    args = _abi(w, fv.FV_FP64)
    q0 = torch.from_numpy(q.copy()).cuda()
    qa, qb = torch.empty_like(q0), torch.empty_like(q0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        _noalloc_step(L, args, dt, q0, qa, qb, stream)
        d = rel_field_diff(q0.cpu().numpy(), refs[call])
        assert np.all(d <= TOL[fv.FV_FP64]), (call, d)


def test_noalloc_rejects_aliased_registers():
    """qout may be q0 itself but may not overlap qprev or part of q0"""
    import torch
    w = wl.random_state(n=(16, 12))
    L = fv.load()
    g, cm, e = _abi(w, fv.FV_FP64)
    nbytes = w.nvar * w.cells * 8
    buf = torch.zeros(3 * w.nvar * w.cells, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(k, q0, qprev, qout):
        return L.fv_rk_stage_noalloc(C.byref(g), C.byref(cm), C.byref(e), k, 1e-12, C.c_void_p(q0),
                                     C.c_void_p(qprev), C.c_void_p(qout), stream)
    assert call(1, base, base, base) == fv.FV_ERR_ARG                          # qout == qprev (k = 1)
    assert call(2, base, base + nbytes, base + nbytes) == fv.FV_ERR_ARG        # qout == qprev
    assert call(2, base, base + nbytes, base + nbytes + 8) == fv.FV_ERR_ARG    # partial overlap of qprev
    assert call(2, base + 8, base + 2 * nbytes, base) == fv.FV_ERR_ARG        # partial overlap of q0


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    w = wl.random_state(n=(2048, 2048))
    L = fv.load()
    g, cm, e = _abi(w, fv.FV_FP64)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    st = L.fv_rk_stage_noalloc(C.byref(g), C.byref(cm), C.byref(e), 1, 1e-9, p, p, p,
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fv.FV_ERR_ARG
