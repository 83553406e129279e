"""The binding's marshalling of a workload into the C structs (no GPU): every
field of fv_grid, fv_components and fv_eos carries the workload's value of
the same name.  Each field gets a distinct value, so a swapped or
positional mix-up fails; the oracle's own marshalling (written apart from
the binding) carries the same values."""
import dataclasses

from paper_2304_00140_gb300 import fv, workloads as wl

import oracle

COMP_FIELDS = ("kind", "gamma", "pinf", "cv", "q", "Tc", "pc", "omega", "M", "mu", "kc", "psat", "rho_sl",
               "rho_sv", "cl", "rt")
EOS_FIELDS = ("beta", "thinc_eps", "thinc_gamma", "thr_ducros", "thr_gas", "eps_ducros", "d3p_coef", "sigma",
              "grad_eps", "thr_vap")
ORACLE_EOS = {"beta": "beta", "thinc_eps": "thinc_eps", "thinc_gamma": "thinc_gamma", "thr_ducros": "thr_ducros",
              "thr_gas": "thr_gas", "eps_ducros": "eps_ducros", "d3p_coef": "d3p_coef", "sigma": "sigma",
              "grad_eps": "grad_eps", "thr_vap": "thr_vap"}


def _workload():
    comps = []
    for k in range(3):
        c = {f: 1.0 + 0.01 * i + 0.1 * k for i, f in enumerate(COMP_FIELDS)}
        c["kind"] = 0
        comps.append(c)
    scheme = wl.default_scheme(iles=1, thinc=1, lim_vel=2, lim_scalar=5, precision=1, curvature=1, st_model=1,
                               gravity=(0.1, -9.8, 0.3), p_ref=3.3e5, T_ref=311.0)
    for i, f in enumerate(EOS_FIELDS):
        scheme[f] = 0.5 + 0.03 * i
    w = wl.jet3d(n=(8, 6, 5))
    inflow = dict(yc=1.1e-3, zc=0.9e-3, radius=0.3e-3, T=351.0, Y=[0.15, 0.25], u0=(250.0, 3.0, -4.0))
    return dataclasses.replace(w, comps=comps, scheme=scheme, inflow=inflow, lo=[0.1e-3, 0.2e-3, 0.3e-3],
                               hi=[4.1e-3, 2.2e-3, 2.3e-3], bc=[[3, 2], [1, 2], [0, 0]])


def test_structs_carry_the_workloads_values():
    w = _workload()
    g, cm, e = fv.make_grid(w), fv.make_components(w), fv.make_eos(w.scheme)
    assert g.ndim == 3
    for d in range(3):
        assert (g.n[d], g.lo[d], g.hi[d], g.bc[d][0], g.bc[d][1]) == (w.n[d], w.lo[d], w.hi[d], *w.bc[d])
    f = w.inflow
    assert (g.in_yc, g.in_zc, g.in_radius, g.in_T) == (f["yc"], f["zc"], f["radius"], f["T"])
    assert list(g.in_u0) == list(f["u0"]) and list(g.in_Y)[:2] == f["Y"]
    assert cm.ncomp == 3 and cm.liquid == w.liquid
    for k, c in enumerate(w.comps):
        for name in COMP_FIELDS:
            assert getattr(cm.comp[k], name) == c[name], (k, name)
    s = w.scheme
    for name in EOS_FIELDS + ("p_ref", "T_ref"):
        assert getattr(e, name) == s[name], name
    for name in ("iles", "thinc", "lim_vel", "lim_scalar", "precision", "curvature", "st_model"):
        assert getattr(e, name) == s[name], name
    assert list(e.gravity) == list(s["gravity"])


def test_binding_and_oracle_marshal_alike():
    w = _workload()
    g, cm, e = fv.make_grid(w), fv.make_components(w), fv.make_eos(w.scheme)
    P = oracle.make_params(w)
    for d in range(3):
        assert P.n[d] == g.n[d] and P.bc[d][0] == g.bc[d][0] and P.bc[d][1] == g.bc[d][1]
        assert abs(P.dx[d] - (g.hi[d] - g.lo[d]) / g.n[d]) <= 1e-15 * P.dx[d]
    # the oracle keeps the disc centre relative to the box corner
    assert abs(P.in_yc - (g.in_yc - g.lo[1])) < 1e-18 and abs(P.in_zc - (g.in_zc - g.lo[2])) < 1e-18
    assert (P.in_radius, P.in_T) == (g.in_radius, g.in_T)
    assert list(P.in_u0) == list(g.in_u0) and list(P.in_Y)[:2] == list(g.in_Y)[:2]
    assert P.ncomp == cm.ncomp and P.liquid == cm.liquid
    for k in range(3):
        for name in COMP_FIELDS:
            assert getattr(P.comp[k], name) == getattr(cm.comp[k], name), (k, name)
    for fname, pname in ORACLE_EOS.items():
        assert getattr(P, pname) == getattr(e, fname), fname
    assert (P.iles, P.thinc, P.lim_vel, P.lim_scalar) == (e.iles, e.thinc, e.lim_vel, e.lim_scalar)
    assert (P.curv, P.st_model) == (e.curvature, e.st_model)
    assert list(P.grav) == list(e.gravity)
