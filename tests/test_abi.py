"""The C-ABI library builds, loads and exports every symbol include/thinc_fv.h
declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2304_00140_gb300 import fv, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "thinc_fv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = fv.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(fv.EXPORTS) == names


def test_workspace_size_and_argument_checks():
    L = fv.load()
    w = wl.advection(n=32)
    g = (fv.fv_grid * 1)(fv.make_grid(w))
    cm, e = fv.make_components(w), fv.make_eos(w.scheme)
    n = C.c_size_t()
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_OK
    # three FP64 registers of 5 fields plus primitives at least
    assert n.value >= 3 * 5 * 32 * 32 * 8 + 5 * 36 * 36 * 8
    bad = fv.make_grid(w)
    bad.n[0] = 0
    assert L.fv_workspace_size(1, (fv.fv_grid * 1)(bad), C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    bad = fv.make_grid(w)
    bad.bc[0][1] = wl.BC_OUTFLOW          # periodic paired with outflow
    assert L.fv_workspace_size(1, (fv.fv_grid * 1)(bad), C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    ctx = C.c_void_p()
    e2 = fv.make_eos(dict(w.scheme, lim_vel=9))
    st = L.fv_init(1, g, C.byref(cm), C.byref(e2), C.byref(ctx))
    assert st == fv.FV_ERR_ARG
    assert b"limiter" in L.fv_last_error(ctx)
    L.fv_destroy(ctx)
    cm3 = fv.make_components(w)
    cm3.comp[0].pinf = 1e7                 # three distinct pinf values
    cm3.ncomp = 3
    cm3.comp[2] = fv.fv_component(0, 2.0, 5e8, 1000.0, 0, 0, 0, 0, 0)
    assert L.fv_workspace_size(1, g, C.byref(cm3), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    assert L.fv_status_string(fv.FV_ERR_NONPHYSICAL) == b"FV_ERR_NONPHYSICAL"


def test_peng_robinson_argument_checks():
    L = fv.load()
    w = wl.pr_shock_droplet(n=32)
    g = (fv.fv_grid * 1)(fv.make_grid(w))
    cm, e = fv.make_components(w), fv.make_eos(w.scheme)
    n = C.c_size_t()
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_OK
    e2 = fv.make_eos(dict(w.scheme, sigma=0.07))          # CSF needs volume fractions: SG/IG only
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e2), C.byref(n)) == fv.FV_ERR_ARG
    cm2 = fv.make_components(w)
    cm2.comp[0] = fv.fv_component(0, 1.4, 0.0, 718.0, 0, 0, 0, 0, 0)   # SG mixed with PR
    assert L.fv_workspace_size(1, g, C.byref(cm2), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG


def test_viscous_and_gravity_argument_checks():
    L = fv.load()
    n = C.c_size_t()
    w = wl.rising_bubble(1, n=(20, 40))
    g = (fv.fv_grid * 1)(fv.make_grid(w))
    cm, e = fv.make_components(w), fv.make_eos(w.scheme)
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_OK
    w0 = wl.with_transport(w, mu=[0.0, 0.0], gravity=(0.0, 0.0, 0.0))
    n0 = C.c_size_t()
    assert L.fv_workspace_size(1, g, C.byref(fv.make_components(w0)), C.byref(fv.make_eos(w0.scheme)),
                               C.byref(n0)) == fv.FV_OK
    assert n.value > n0.value          # rho, c (gravity) and mu, k_c (viscosity) primitive fields
    bad = fv.make_components(w)
    bad.comp[0].mu = -1.0
    assert L.fv_workspace_size(1, g, C.byref(bad), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    bad = fv.make_components(w)
    bad.comp[1].kc = float("nan")
    assert L.fv_workspace_size(1, g, C.byref(bad), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    e2 = fv.make_eos(w.scheme)
    e2.gravity[1] = float("inf")
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e2), C.byref(n)) == fv.FV_ERR_ARG
    # Peng-Robinson mixtures have no volume fractions for Eq. 2-8
    wp = wl.pr_shock_droplet(n=32)
    gp = (fv.fv_grid * 1)(fv.make_grid(wp))
    cmp_ = fv.make_components(wl.with_transport(wp, mu=[1e-5, 1e-3]))
    assert L.fv_workspace_size(1, gp, C.byref(cmp_), C.byref(fv.make_eos(wp.scheme)), C.byref(n)) == fv.FV_ERR_ARG


def test_struct_layout_matches_header(tmp_path):
    """offsets and sizes of the ABI structs as the C compiler lays them out
    from include/thinc_fv.h equal the ctypes mirrors of the binding"""
    structs = {"fv_grid": fv.fv_grid, "fv_component": fv.fv_component, "fv_components": fv.fv_components,
               "fv_eos": fv.fv_eos}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "thinc_fv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for f in cls._fields_:
            assert int(out[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


def test_barotropic_argument_checks():
    L = fv.load()
    n = C.c_size_t()
    w = wl.bubble_collapse("vapour", n=(20, 20))
    g = (fv.fv_grid * 1)(fv.make_grid(w))
    e = fv.make_eos(w.scheme)
    assert L.fv_workspace_size(1, g, C.byref(fv.make_components(w)), C.byref(e), C.byref(n)) == fv.FV_OK
    for field, val in (("rho_sv", 2000.0), ("cl", 0.0), ("psat", -1.0)):
        cm = fv.make_components(w)
        setattr(cm.comp[w.liquid], field, val)
        assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG, field
    cm = fv.make_components(w)
    cm.comp[0].rt = 0.0                                   # a gas without R T_ref
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
    cm = fv.make_components(w)
    cm.comp[0] = fv.make_components(wl.advection(n=8)).comp[0]   # a stiffened gas among barotropic ones
    assert L.fv_workspace_size(1, g, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG


def test_noalloc_host_side_argument_checks():
    """fv_rk_stage_noalloc rejects, before any device work, what fv_init
    rejects, extents whose ghosted sizes would overflow, and output arrays
    that overlap its inputs (the pointers here are never dereferenced)"""
    L = fv.load()
    w = wl.random_state(n=(16, 12))
    g, cm, e = fv.make_grid(w), fv.make_components(w), fv.make_eos(w.scheme)
    nbytes = w.nvar * w.cells * 8
    base = 1 << 40

    def call(grid, k, q0, qprev, qout, eos=e):
        return L.fv_rk_stage_noalloc(C.byref(grid), C.byref(cm), C.byref(eos), k, 1e-12, C.c_void_p(q0),
                                     C.c_void_p(qprev), C.c_void_p(qout), None)
    assert call(g, 1, base, base, base) == fv.FV_ERR_ARG                         # qout == qprev
    assert call(g, 2, base, base + nbytes, base + nbytes + 8) == fv.FV_ERR_ARG   # overlaps qprev
    assert call(g, 2, base + 8, base + 2 * nbytes, base) == fv.FV_ERR_ARG       # overlaps part of q0
    assert call(g, 0, base, base + nbytes, base + 2 * nbytes) == fv.FV_ERR_ARG   # stage index
    for n in ((2 ** 31 - 2, 2), (2 ** 16, 2 ** 16), (70000, 70000)):
        big = fv.make_grid(w)
        big.n[0], big.n[1] = n
        assert call(big, 1, base, base, base + nbytes) == fv.FV_ERR_ARG
    e2 = fv.make_eos(dict(w.scheme, gravity=(float("nan"), 0.0, 0.0)))
    assert call(g, 2, base, base + nbytes, base + 2 * nbytes, eos=e2) == fv.FV_ERR_ARG


def test_split_host_side_argument_checks():
    """fv_split_workspace_size checks the slab plan without a device: at
    least two planes per slab, plane counts adding up to the grid's extent;
    a valid split needs a little more memory than the unsplit grid (the
    slabs' ghost planes in every conserved register)"""
    L = fv.load()
    w = wl.random_state(n=(16, 12))
    g, cm, e = fv.make_grid(w), fv.make_components(w), fv.make_eos(w.scheme)
    n0, n = C.c_size_t(), C.c_size_t()
    assert L.fv_workspace_size(1, (fv.fv_grid * 1)(g), C.byref(cm), C.byref(e), C.byref(n0)) == fv.FV_OK
    rows = lambda *r: (C.c_int * len(r))(*r)
    assert L.fv_split_workspace_size(C.byref(g), 2, None, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_OK
    assert n.value > n0.value
    assert L.fv_split_workspace_size(C.byref(g), 3, rows(4, 4, 4), C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_OK
    for nb, r in ((2, rows(5, 6)), (3, rows(1, 5, 6)), (7, None), (0, None)):
        assert L.fv_split_workspace_size(C.byref(g), nb, r, C.byref(cm), C.byref(e), C.byref(n)) == fv.FV_ERR_ARG
