"""The z-marching 3D stage kernel (FP32-mixed form) against the tiled stage
kernel and against the FP64 oracle.  The two kernels evaluate the same
formulas in the same order (sensor, smoothed fraction, vertex normals,
faces, curvature, update), organised per z-plane or per 3D tile, so their
results agree to rounding; the oracle bounds the mixed form's error."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import rel_field_diff, rel_l1_vec

pytestmark = pytest.mark.gpu


def _run(w, kernel, monkeypatch, steps=2, inflow_u=None, zvar=None):
    monkeypatch.setenv("FV_ZMARCH", "1" if kernel == "zmarch" else "0")
    if zvar is None:
        monkeypatch.delenv("FV_ZVAR", raising=False)
    else:
        monkeypatch.setenv("FV_ZVAR", str(zvar))
    s = fv.Solver(w, precision=fv.FV_MIXED, inflow_u=[inflow_u] if inflow_u is not None else None)
    q = oracle.Oracle(w, inflow_u=inflow_u).prim_to_cons(w.primitives())
    s.set_state(q)
    s.step(steps, w.cfl)
    t = s.tile()
    assert t["zmarch"] == (kernel == "zmarch")
    if zvar is not None:
        assert t["fused_variant"] == zvar and t["threads"] == ZVAR_THREADS[zvar]
    return q, s.get_state()


# the z-marching kernel's variants with the Table 4.2 limiter pair and their block sizes
ZVAR_THREADS = {0: 320, 1: 256, 3: 352, 4: 416, 5: 288}


CASES = {
    "plain_2comp": lambda: wl.random_state(n=(37, 22, 19), ndim=3, ncomp=2),
    "plain_3comp_bc": lambda: wl.random_state(
        n=(20, 33, 11), ndim=3, ncomp=3,
        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2]),
    "other_limiters": lambda: wl.random_state(n=(21, 18, 13), ndim=3, ncomp=2, iles=1,
                                              lim_vel=wl.LIM_VANLEER, lim_scalar=wl.LIM_MC),
    "iles_csf_3comp": lambda: wl.random_state(
        n=(18, 17, 40), ndim=3, ncomp=3, iles=1, sigma=5.0,
        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_PERIODIC] * 2, [wl.BC_REFLECT, wl.BC_OUTFLOW]]),
    # Eq. 2-2 viscous stresses, heat flux and gravity (the kernel's viscous instantiations)
    "visc_grav_2comp_bc": lambda: wl.with_transport(
        wl.random_state(n=(21, 18, 23), ndim=3, ncomp=2,
                        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2]),
        mu=[2e-3, 5e-3], kc=[0.4, 0.6], gravity=(0.3, -9.8, 0.2)),
    "visc_grav_iles_csf_3comp": lambda: wl.with_transport(
        wl.random_state(n=(18, 17, 21), ndim=3, ncomp=3, iles=1, sigma=5.0,
                        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_PERIODIC] * 2, [wl.BC_REFLECT, wl.BC_OUTFLOW]]),
        mu=[2e-3, 5e-3, 1e-3], kc=[0.4, 0.6, 0.1], gravity=(0.3, -9.8, 0.2)),
    "visc_runtime_limiters": lambda: wl.with_transport(
        wl.random_state(n=(19, 16, 14), ndim=3, ncomp=2, lim_vel=wl.LIM_VANLEER, lim_scalar=wl.LIM_MC),
        mu=[40.0, 80.0], kc=[0.0, 0.0], gravity=(0.0, 0.0, 0.0)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_zmarch_matches_tiled_kernel(name, monkeypatch):
    w = CASES[name]()
    _, a = _run(w, "zmarch", monkeypatch)
    _, b = _run(w, "tiled", monkeypatch)
    d = rel_field_diff(a, b)
    assert np.all(d < 1e-6), d


@pytest.mark.parametrize("zvar", sorted(ZVAR_THREADS))
@pytest.mark.parametrize("name", ["plain_3comp_bc", "iles_csf_3comp"])
def test_zmarch_variants_match_tiled_kernel(name, zvar, monkeypatch):
    """every block size of the z-marching kernel (its face tasks and sensor
    cells spread over 8 to 13 warps) against the tiled kernel"""
    w = CASES[name]()
    _, a = _run(w, "zmarch", monkeypatch, zvar=zvar)
    _, b = _run(w, "tiled", monkeypatch)
    d = rel_field_diff(a, b)
    assert np.all(d < 1e-6), d


def test_zmarch_jet_inflow_matches_tiled_kernel(monkeypatch):
    w = wl.jet3d(n=(40, 24, 24))
    w.inflow["radius"] = 5.5 * w.dx[1]
    u = wl.jet_inflow_velocity(w)
    _, a = _run(w, "zmarch", monkeypatch, steps=3, inflow_u=u)
    _, b = _run(w, "tiled", monkeypatch, steps=3, inflow_u=u)
    d = rel_field_diff(a, b)
    assert np.all(d < 1e-6), d


def test_zmarch_mixed_accuracy_against_oracle(monkeypatch):
    """App. D + CSF, three components: relative L1 per conserved field of the
    mixed z-marching run against the FP64 oracle after two steps."""
    w = CASES["iles_csf_3comp"]()
    q, got = _run(w, "zmarch", monkeypatch)
    ref, _ = oracle.Oracle(w).step(q, 2, w.cfl)
    e = rel_l1_vec(got, ref, w.ndim)
    assert np.all(e < 1e-4), e


FP64_CASES = ["plain_2comp", "plain_3comp_bc", "other_limiters", "iles_csf_3comp"]


@pytest.mark.parametrize("zvar", [None, 1, 4, 5])
@pytest.mark.parametrize("name", FP64_CASES)
def test_zmarch_fp64_parity_with_oracle(name, zvar, monkeypatch):
    """the z-marching kernel in the FP64 form (double plane ring, one block
    per SM; the tuner's variant, or 256 / 416 / 288 threads) against the FP64
    oracle: three steps of 0.3 x the oracle's CFL step, 1e-10 of each
    field's scale (momentum against the momentum vector's)"""
    from tests.helpers import oracle_step_dt
    if zvar is not None and name == "other_limiters":
        pytest.skip("the run-time limiter pair has one FP64 variant (2)")
    monkeypatch.setenv("FV_ZMARCH", "1")
    if zvar is None:
        monkeypatch.delenv("FV_ZVAR", raising=False)
    else:
        monkeypatch.setenv("FV_ZVAR", str(zvar))
    w = CASES[name]()
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    ref = q
    for _ in range(3):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
    assert s.tile()["zmarch"]
    if zvar is not None:
        assert s.tile()["fused_variant"] == zvar and s.tile()["threads"] == ZVAR_THREADS[zvar]
    got = s.get_state()
    d = rel_field_diff(got, ref)
    mag = np.sqrt((ref[1:4] ** 2).sum(0)).max()
    for a in range(3):
        d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    assert np.all(d < 1e-10), d


def test_zmarch_fp64_jet_inflow_parity(monkeypatch):
    """FP64 z-march on the jet with per-cell inflow velocities, App. D and
    CSF, against the oracle (two steps)"""
    from tests.helpers import oracle_step_dt
    monkeypatch.setenv("FV_ZMARCH", "1")
    w = wl.jet3d(n=(40, 24, 24))
    w.inflow["radius"] = 5.5 * w.dx[1]
    u = wl.jet_inflow_velocity(w)
    o = oracle.Oracle(w, inflow_u=u)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64, inflow_u=[u])
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    ref = q
    for _ in range(2):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
    assert s.tile()["zmarch"]
    got = s.get_state()
    d = rel_field_diff(got, ref)
    mag = np.sqrt((ref[1:4] ** 2).sum(0)).max()
    for a in range(3):
        d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    assert np.all(d < 1e-10), d
