"""Shared helpers of the tests: building contexts and comparing fields."""
import numpy as np

import oracle

LSRK_STAGES = (1, 2, 3, 4)


def rel_field_diff(a, b):
    """max |a - b| / max |b| per field (first axis)."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return np.abs(a - b).max(axis=1) / scale


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.abs(a - b).sum(axis=1) / np.maximum(np.abs(b).sum(axis=1), 1e-300)


def oracle_step_dt(o, q, dt):
    """one full LSRK step of the oracle with a given dt"""
    q0 = np.ascontiguousarray(q)
    qa = o.stage(1, dt, q0, q0)
    qb = o.stage(2, dt, q0, qa)
    qa = o.stage(3, dt, q0, qb)
    return o.stage(4, dt, q0, qa)


def oracle_step_window(o, q, dt, lo, hi):
    """one LSRK step of the oracle on the window [lo, hi) only: stage k is
    evaluated on the window grown by 2 (4 - k) cells (clipped to the domain),
    which is all that stage k + 1 reads.  Returns the full array with the
    window filled in.  Exact where the grown window does not cross a periodic
    side (walls, outflow and inflow sides are fine): the growth is clipped,
    not wrapped.  With the capillary jump a face also reads the curvature of
    its two cells, which reaches two cells further, so a stage reads three
    cells on each side and the growth is 3 (4 - k)."""
    w = o.w
    q0 = np.ascontiguousarray(q)
    prev = q0
    reach = 3 if (w.scheme.get("st_model", 0) == 1 and w.scheme.get("sigma", 0.0) > 0.0) else 2
    for k in LSRK_STAGES:
        g = reach * (4 - k)
        wl_ = [max(0, lo[d] - g) if d < w.ndim else 0 for d in range(3)]
        wh_ = [min(w.n[d], hi[d] + g) if d < w.ndim else 1 for d in range(3)]
        out = q0.copy()
        o.stage(k, dt, q0, prev, window=(wl_, wh_), out=out)
        prev = out
    return prev


def rel_l1_vec(a, b, ndim):
    """relative L1 per conserved field; the momentum components are measured
    against the L1 norm of the momentum vector (a component can be ~0)"""
    nv = a.shape[0]
    den = np.abs(b).reshape(nv, -1).sum(1)
    den[1:1 + ndim] = np.sqrt((b[1:1 + ndim] ** 2).sum(0)).sum()
    return np.abs(a - b).reshape(nv, -1).sum(1) / np.maximum(den, 1e-300)


def gpu_stage(w, precision, k, dt, q0, qprev):
    """one stage q0 + a_k dt R(qprev) of workload w on the GPU through the
    C ABI's fv_rk_stage_noalloc, from host arrays (the tiled stage kernel)"""
    import ctypes as C

    import torch

    from paper_2304_00140_gb300 import fv
    L = fv.load()
    g, cm = fv.make_grid(w), fv.make_components(w)
    e = fv.make_eos(dict(w.scheme, precision=precision))
    d0 = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    dp = torch.from_numpy(np.ascontiguousarray(qprev)).cuda()
    out = torch.empty_like(d0)
    st = L.fv_rk_stage_noalloc(C.byref(g), C.byref(cm), C.byref(e), k, dt, C.c_void_p(d0.data_ptr()),
                               C.c_void_p(dp.data_ptr()), C.c_void_p(out.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fv.FV_OK, fv.status_string(st)
    return out.cpu().numpy()


def cell_rel_diff(a, b):
    """per cell, the largest over fields of |a - b| / max |b| of the field"""
    nv = a.shape[0]
    scale = np.maximum(np.abs(b).reshape(nv, -1).max(axis=1), 1e-300)
    return (np.abs(a - b) / scale.reshape((nv,) + (1,) * (a.ndim - 1))).max(axis=0)
